/*
 * FP64 CPU oracle for the GS-LIVO differentiable Gaussian-splatting path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the renderer computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg call it.  It shares no code,
 * header, constant table or helper with the CUDA library and includes nothing
 * from it.
 *
 * Everything is double precision.  Each function cites the passage of the
 * paper it restates:
 *   - Sec. II-B.1, Eq. 3dgs:        Sigma3 = (R S)(R S)^T
 *   - Sec. II-B.1, Eq. q:           q_i = pi(T_CW p_W)
 *   - Sec. II-B.1, Eq. spat:        Sigma2 = (J W) Sigma3 (J W)^T, W = R_CW
 *   - Sec. II-B.2, Eq. raster:      front-to-back alpha compositing
 *   - Sec. II-B.2, Eq. gaussian_optimization and Sec. II-D,
 *     Eq. minimization:             photometric loss, minimised over the
 *                                   Gaussian parameters and over the pose
 *   - Appendix A, perturbation model: left perturbation of T_CW
 *   - Sec. II-D, Eq. minimization: the per-pixel pose Jacobian of the
 *                                   rendered image (measurement Jacobian of
 *                                   the photometric update) and its normal
 *                                   equations
 *   - Sec. II-B.2 ("Adam optimizer"): Kingma-Ba Adam with bias correction.
 *
 * Readings taken where the paper is silent (the same ones the CUDA path uses):
 *   - alpha_i(x) = sigma_i G_i(x), every G evaluated at the pixel x;
 *   - alpha is clamped to alpha_max; a Gaussian with alpha < alpha_min is
 *     skipped; compositing stops before the Gaussian that would take the
 *     transmittance below T_min;
 *   - a low-pass blur b is added to the diagonal of Sigma2;
 *   - pixel (u, v) is sampled at (u + 0.5, v + 0.5);
 *   - depth ties are ordered by Gaussian index;
 *   - colour = max(0, sum_k Y_k(d) k_k + 0.5) with d the unit view direction
 *     from the camera centre and Y_k, k = l^2 + l + m, the real spherical
 *     harmonics of degree l <= 3 with the Condon-Shortley phase, ordered
 *     m = -l..l (degree 1: Y = C1 (-d_y, d_z, -d_x));
 *   - opacity sigma = sigmoid(logit); scale = exp(log-scale);
 *   - clamps contribute zero derivative; culling is locally constant.
 * With alpha_min = 0, alpha_max = 1, T_min = 0 ("exact mode") the compositing
 * is literally Eq. raster over every Gaussian in front of the camera.
 *
 * cfg[] layout (doubles): alpha_min, alpha_max, T_min, blur, z_near,
 *                         bg_r, bg_g, bg_b.
 * cam[] layout (doubles): R_CW (9, row-major), t_CW (3), fx, fy, cx, cy.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* Host threads of the parallel loops: n_threads > 0 for one call, otherwise
 * the process-wide count set by orc_set_num_threads (all processors by
 * default).  Threads only split independent pixels or Gaussians; every sum
 * over threads is taken in thread order. */
static int orc_default_threads = 0;

static int orc_threads(int n_threads) {
    if (n_threads > 0) return n_threads;
    if (orc_default_threads > 0) return orc_default_threads;
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) { orc_default_threads = n > 0 ? n : 0; }

/* Unit roundoff of binary32.  Depth order is decided on the camera depth
 * R_CW[2] . p_W + t_CW[2] of binary32 inputs evaluated as a compensated dot
 * product in binary32 arithmetic ("Dot2", Ogita, Rump and Oishi 2005), whose
 * unevaluated result errs by at most gamma_4^2 sum |terms| with
 * gamma_n = n u / (1 - n u).  Two contributors closer in depth than the sum
 * of their bounds may be ordered either way. */
#define U32 (1.0 / 16777216.0)

/* Real spherical harmonics up to degree 3 at the direction d (a unit
 * vector), with the Condon-Shortley phase (-1)^m, index k = l^2 + l + m,
 * written as homogeneous polynomials of degree l in (x, y, z) = d (on the
 * unit sphere r^2 = 1 completes the textbook forms, e.g. 5 z^2 - 3 r^2), and
 * their partial derivatives dY[k][j] = dY_k / dd_j of those polynomials.
 * Normalisations, from N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the
 * associated Legendre factor (x sqrt 2 for m != 0):
 *   l = 0: 1/2 sqrt(1/pi);  l = 1: 1/2 sqrt(3/pi);
 *   l = 2: 1/2 sqrt(15/pi) (xy, yz, xz), 1/4 sqrt(5/pi) (2z^2 - x^2 - y^2),
 *          1/4 sqrt(15/pi) (x^2 - y^2);
 *   l = 3: 1/4 sqrt(35/(2 pi)) (y (3x^2 - y^2), x (x^2 - 3y^2)),
 *          1/2 sqrt(105/pi) (xyz), 1/4 sqrt(21/(2 pi)) (y, x times
 *          4z^2 - x^2 - y^2), 1/4 sqrt(7/pi) (z (2z^2 - 3x^2 - 3y^2)),
 *          1/4 sqrt(105/pi) (z (x^2 - y^2)). */
static void sh_basis(const double* d, int degree, double* Y, double dY[16][3]) {
    double x = d[0], y = d[1], z = d[2];
    for (int k = 0; k < 16; ++k) {
        Y[k] = 0.0;
        dY[k][0] = dY[k][1] = dY[k][2] = 0.0;
    }
    Y[0] = 0.5 * sqrt(1.0 / ORC_PI);
    if (degree < 1) return;
    double c1 = 0.5 * sqrt(3.0 / ORC_PI);
    Y[1] = -c1 * y; dY[1][1] = -c1;
    Y[2] = c1 * z;  dY[2][2] = c1;
    Y[3] = -c1 * x; dY[3][0] = -c1;
    if (degree < 2) return;
    double a = 0.5 * sqrt(15.0 / ORC_PI), b = 0.25 * sqrt(5.0 / ORC_PI), c = 0.25 * sqrt(15.0 / ORC_PI);
    Y[4] = a * x * y;
    dY[4][0] = a * y; dY[4][1] = a * x;
    Y[5] = -a * y * z;
    dY[5][1] = -a * z; dY[5][2] = -a * y;
    Y[6] = b * (2.0 * z * z - x * x - y * y);
    dY[6][0] = -2.0 * b * x; dY[6][1] = -2.0 * b * y; dY[6][2] = 4.0 * b * z;
    Y[7] = -a * x * z;
    dY[7][0] = -a * z; dY[7][2] = -a * x;
    Y[8] = c * (x * x - y * y);
    dY[8][0] = 2.0 * c * x; dY[8][1] = -2.0 * c * y;
    if (degree < 3) return;
    double e = 0.25 * sqrt(35.0 / (2.0 * ORC_PI)), f = 0.5 * sqrt(105.0 / ORC_PI);
    double g = 0.25 * sqrt(21.0 / (2.0 * ORC_PI)), h = 0.25 * sqrt(7.0 / ORC_PI);
    double j = 0.25 * sqrt(105.0 / ORC_PI);
    Y[9] = -e * y * (3.0 * x * x - y * y);
    dY[9][0] = -6.0 * e * x * y; dY[9][1] = -e * (3.0 * x * x - 3.0 * y * y);
    Y[10] = f * x * y * z;
    dY[10][0] = f * y * z; dY[10][1] = f * x * z; dY[10][2] = f * x * y;
    Y[11] = -g * y * (4.0 * z * z - x * x - y * y);
    dY[11][0] = 2.0 * g * x * y; dY[11][1] = -g * (4.0 * z * z - x * x - 3.0 * y * y);
    dY[11][2] = -8.0 * g * y * z;
    Y[12] = h * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    dY[12][0] = -6.0 * h * x * z; dY[12][1] = -6.0 * h * y * z;
    dY[12][2] = h * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    Y[13] = -g * x * (4.0 * z * z - x * x - y * y);
    dY[13][0] = -g * (4.0 * z * z - 3.0 * x * x - y * y); dY[13][1] = 2.0 * g * x * y;
    dY[13][2] = -8.0 * g * x * z;
    Y[14] = j * z * (x * x - y * y);
    dY[14][0] = 2.0 * j * x * z; dY[14][1] = -2.0 * j * y * z; dY[14][2] = j * (x * x - y * y);
    Y[15] = -e * x * (x * x - 3.0 * y * y);
    dY[15][0] = -e * (3.0 * x * x - 3.0 * y * y); dY[15][1] = 6.0 * e * x * y;
}

/* The basis above for n directions (tests): Y [n][16], dY [n][16][3]. */
int orc_sh_basis(long n, const double* dirs, int degree, double* Y, double* dY) {
    if (degree < 0 || degree > 3) return -1;
    for (long i = 0; i < n; ++i) {
        double y[16], dy[16][3];
        sh_basis(dirs + 3 * i, degree, y, dy);
        for (int k = 0; k < 16; ++k) {
            Y[16 * i + k] = y[k];
            for (int c = 0; c < 3; ++c) dY[48 * i + 3 * k + c] = dy[k][c];
        }
    }
    return 0;
}

/* Rotation of the unit quaternion (w, x, y, z): the textbook formula. */
static void quat_to_R(const double* qh, double* R) {
    double w = qh[0], x = qh[1], y = qh[2], z = qh[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Everything the forward projection of one Gaussian produces, kept so that the
 * backward pass can walk the same chain in reverse. */
typedef struct {
    int valid;
    double qn;        /* |quat| */
    double qh[4];     /* unit quaternion */
    double R[9];      /* R(qh) */
    double sc[3];     /* exp(log-scale) */
    double M[9];      /* R S */
    double S3[9];     /* Sigma3 = M M^T */
    double pc[3];     /* camera-frame mean */
    double zerr;      /* bound on the FP32 rounding error of pc[2] */
    double J[6];      /* 2x3 projection Jacobian */
    double T[6];      /* J W */
    double S2[3];     /* Sigma2 = T Sigma3 T^T + b I: (a, b, c) */
    double conic[3];  /* Sigma2^-1: (A, B, C) */
    double q[2];      /* projected mean (pixels) */
    double sigma;     /* opacity */
    double dvec[3];   /* mu - campos */
    double dlen;
    double dir[3];    /* unit view direction */
    double raw[3];    /* colour before the clamp */
    double colour[3];
} orc_proj;

/* Projection of Gaussian i into camera `cam` (Eqs. 3dgs, q, spat). */
static void project_one(const double* mu, const double* ls, const double* quat, double ologit,
                        const double* sh, int sh_degree, const double* cam, const double* cfg,
                        orc_proj* P) {
    const double* W = cam;       /* R_CW */
    const double* t = cam + 9;   /* t_CW */
    double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    double blur = cfg[3], z_near = cfg[4];
    memset(P, 0, sizeof(*P));

    /* Sigma3 = (R S)(R S)^T with S = diag(exp(s)) (Eq. 3dgs). */
    P->qn = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    for (int k = 0; k < 4; ++k) P->qh[k] = quat[k] / P->qn;
    quat_to_R(P->qh, P->R);
    for (int k = 0; k < 3; ++k) P->sc[k] = exp(ls[k]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P->M[3 * i + j] = P->R[3 * i + j] * P->sc[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += P->M[3 * i + k] * P->M[3 * j + k];
            P->S3[3 * i + j] = s;
        }

    /* Camera-frame mean p_C = R_CW p_W + t_CW (Eq. q). */
    for (int i = 0; i < 3; ++i)
        P->pc[i] = W[3 * i] * mu[0] + W[3 * i + 1] * mu[1] + W[3 * i + 2] * mu[2] + t[i];
    {
        double g4 = 4.0 * U32 / (1.0 - 4.0 * U32);
        P->zerr = g4 * g4 * (fabs(W[6] * mu[0]) + fabs(W[7] * mu[1]) + fabs(W[8] * mu[2]) + fabs(t[2]));
    }
    double x = P->pc[0], y = P->pc[1], z = P->pc[2];
    if (!(z > z_near)) { P->valid = 0; return; }

    /* Pinhole projection pi and its Jacobian J (Eq. q, Eq. spat). */
    P->q[0] = fx * x / z + cx;
    P->q[1] = fy * y / z + cy;
    P->J[0] = fx / z; P->J[1] = 0.0;    P->J[2] = -fx * x / (z * z);
    P->J[3] = 0.0;    P->J[4] = fy / z; P->J[5] = -fy * y / (z * z);
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += P->J[3 * r + k] * W[3 * k + c];
            P->T[3 * r + c] = s;
        }
    /* Sigma2 = T Sigma3 T^T + b I (Eq. spat plus the low-pass blur). */
    double S2f[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) s += P->T[3 * r + i] * P->S3[3 * i + j] * P->T[3 * c + j];
            S2f[2 * r + c] = s;
        }
    P->S2[0] = S2f[0] + blur;
    P->S2[1] = 0.5 * (S2f[1] + S2f[2]);
    P->S2[2] = S2f[3] + blur;
    double det = P->S2[0] * P->S2[2] - P->S2[1] * P->S2[1];
    if (!(det > 0.0)) { P->valid = 0; return; }
    P->conic[0] = P->S2[2] / det;
    P->conic[1] = -P->S2[1] / det;
    P->conic[2] = P->S2[0] / det;

    P->sigma = 1.0 / (1.0 + exp(-ologit));

    /* Colour from SH of degree <= 3 along the view direction. */
    double campos[3];
    for (int i = 0; i < 3; ++i) campos[i] = -(W[i] * t[0] + W[3 + i] * t[1] + W[6 + i] * t[2]);
    for (int i = 0; i < 3; ++i) P->dvec[i] = mu[i] - campos[i];
    P->dlen = sqrt(P->dvec[0] * P->dvec[0] + P->dvec[1] * P->dvec[1] + P->dvec[2] * P->dvec[2]);
    for (int i = 0; i < 3; ++i) P->dir[i] = P->dvec[i] / P->dlen;
    double Y[16], dY[16][3];
    int K = (sh_degree + 1) * (sh_degree + 1);
    sh_basis(P->dir, sh_degree, Y, dY);
    for (int ch = 0; ch < 3; ++ch) {
        double v = 0.5;
        for (int k = 0; k < K; ++k) v += Y[k] * sh[3 * k + ch];
        P->raw[ch] = v;
        P->colour[ch] = v > 0.0 ? v : 0.0;
    }
    P->valid = 1;
}

/* Public projection: per Gaussian of one view, the quantities the compositing
 * uses.  Arrays are [n, k] row-major; `valid` is 0 for culled Gaussians. */
int orc_project(long n, const double* means, const double* log_scales, const double* quats,
                const double* opacity, const double* sh, int sh_degree, const double* cam,
                const double* cfg, int* valid, double* pc, double* q, double* sigma2,
                double* conic, double* opac, double* colour, double* raw_colour,
                double* depth_err) {
    int K = (sh_degree + 1) * (sh_degree + 1);
    int nthr = orc_threads(0);
    (void)nthr;
    /* Gaussians are independent. */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthr)
#endif
    for (long i = 0; i < n; ++i) {
        orc_proj P;
        project_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, opacity[i], sh + 3 * K * i,
                    sh_degree, cam, cfg, &P);
        valid[i] = P.valid;
        for (int k = 0; k < 3; ++k) pc[3 * i + k] = P.pc[k];
        q[2 * i] = P.q[0]; q[2 * i + 1] = P.q[1];
        for (int k = 0; k < 3; ++k) {
            sigma2[3 * i + k] = P.S2[k];
            conic[3 * i + k] = P.conic[k];
            colour[3 * i + k] = P.colour[k];
            raw_colour[3 * i + k] = P.raw[k];
        }
        opac[i] = P.sigma;
        depth_err[i] = P.zerr;
    }
    return 0;
}

/* ---------- compositing (Eq. raster) ---------- */

typedef struct { double z; long i; } orc_key;

static int key_cmp(const void* a, const void* b) {
    const orc_key* x = (const orc_key*)a;
    const orc_key* y = (const orc_key*)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->i < y->i) ? -1 : (x->i > y->i);
}

/* Valid Gaussians ordered front to back by (depth, index). */
static long depth_order(long n, const int* valid, const double* depth, long* order) {
    orc_key* keys = (orc_key*)malloc(sizeof(orc_key) * (n > 0 ? n : 1));
    long m = 0;
    for (long i = 0; i < n; ++i)
        if (valid[i]) { keys[m].z = depth[i]; keys[m].i = i; ++m; }
    qsort(keys, m, sizeof(orc_key), key_cmp);
    for (long k = 0; k < m; ++k) order[k] = keys[k].i;
    free(keys);
    return m;
}

/* One fragment of the per-pixel list: Gaussian index, its alpha, the
 * unclamped sigma*G, G, the pixel offset d = x - q, and the transmittance
 * in front of it. */
typedef struct { long i; double alpha, araw, G, dx, dy, Tin; } orc_frag;

#define REL_BORDER 1e-5

/* Front-to-back compositing at pixel centre (px, py): fills `frags` with the
 * contributing fragments, returns their count; *Tout is the final
 * transmittance.  *border is set when a threshold decision lies within
 * REL_BORDER (relative) of its cut, so FP32 may decide it the other way. */
static long composite_pixel(double px, double py, long m, const long* order, const double* q,
                            const double* conic, const double* opac, const double* depth,
                            const double* zerr, const double* cfg, orc_frag* frags, double* Tout,
                            int* border, long* n_considered) {
    double amin = cfg[0], amax = cfg[1], Tmin = cfg[2];
    double T = 1.0;
    long nf = 0;
    int bd = 0;
    double zprev = -1.0, eprev = 0.0;
    long k;
    for (k = 0; k < m; ++k) {
        long i = order[k];
        double dx = px - q[2 * i], dy = py - q[2 * i + 1];
        double A = conic[3 * i], B = conic[3 * i + 1], C = conic[3 * i + 2];
        double power = -0.5 * (A * dx * dx + 2.0 * B * dx * dy + C * dy * dy);
        double G = exp(power);
        double araw = opac[i] * G;
        double alpha = araw < amax ? araw : amax;
        if (amin > 0.0 && fabs(araw - amin) <= REL_BORDER * amin) bd = 1;
        if (fabs(araw - amax) <= REL_BORDER * amax) bd = 1;
        if (alpha < amin) continue;
        if (zprev >= 0.0 && fabs(depth[i] - zprev) <= zerr[i] + eprev) bd = 1;
        zprev = depth[i];
        eprev = zerr[i];
        double Tnext = T * (1.0 - alpha);
        if (Tmin > 0.0 && fabs(Tnext - Tmin) <= REL_BORDER * Tmin) bd = 1;
        if (Tnext < Tmin) { ++k; break; }
        frags[nf].i = i; frags[nf].alpha = alpha; frags[nf].araw = araw; frags[nf].G = G;
        frags[nf].dx = dx; frags[nf].dy = dy; frags[nf].Tin = T;
        ++nf;
        T = Tnext;
    }
    *Tout = T;
    *border = bd;
    if (n_considered) *n_considered = k;
    return nf;
}

/* Renders one view.  rgb is [3, H, W]; T_final, n_contrib and borderline are
 * [H, W].  n_contrib counts the contributing Gaussians. */
int orc_render(int W, int H, long n, const int* valid, const double* q, const double* conic,
               const double* opac, const double* colour, const double* depth,
               const double* depth_err, const double* cfg,
               double* rgb, double* T_final, int* n_contrib, unsigned char* borderline,
               int n_threads) {
    long* order = (long*)malloc(sizeof(long) * (n > 0 ? n : 1));
    long m = depth_order(n, valid, depth, order);
    const double* bg = cfg + 5;
    int nthr = orc_threads(n_threads);
    (void)nthr;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthr)
#endif
    {
        orc_frag* frags = (orc_frag*)malloc(sizeof(orc_frag) * (m > 0 ? m : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int v = 0; v < H; ++v) {
            for (int u = 0; u < W; ++u) {
                double T;
                int bd;
                long nf = composite_pixel(u + 0.5, v + 0.5, m, order, q, conic, opac, depth, depth_err, cfg,
                                          frags, &T, &bd, NULL);
                double C[3] = {0.0, 0.0, 0.0};
                for (long f = 0; f < nf; ++f) {
                    long i = frags[f].i;
                    for (int ch = 0; ch < 3; ++ch)
                        C[ch] += colour[3 * i + ch] * frags[f].alpha * frags[f].Tin;
                }
                long pix = (long)v * W + u;
                for (int ch = 0; ch < 3; ++ch) rgb[(long)ch * W * H + pix] = C[ch] + T * bg[ch];
                T_final[pix] = T;
                n_contrib[pix] = (int)nf;
                borderline[pix] = (unsigned char)bd;
            }
        }
        free(frags);
    }
    free(order);
    return 0;
}

/* Eq. raster at a list of pixels (px[k], py[k]) of one view: rgb [n_pix, 3],
 * T_final [n_pix], n_contrib [n_pix], borderline [n_pix].  The same
 * per-pixel compositing as orc_render, for sampled checks of large images. */
int orc_render_pixels(long n_pix, const int* px, const int* py, long n, const int* valid,
                      const double* q, const double* conic, const double* opac,
                      const double* colour, const double* depth, const double* depth_err,
                      const double* cfg, double* rgb,
                      double* T_final, int* n_contrib, unsigned char* borderline, int n_threads) {
    long* order = (long*)malloc(sizeof(long) * (n > 0 ? n : 1));
    long m = depth_order(n, valid, depth, order);
    const double* bg = cfg + 5;
    int nthr = orc_threads(n_threads);
    (void)nthr;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthr)
#endif
    {
        orc_frag* frags = (orc_frag*)malloc(sizeof(orc_frag) * (m > 0 ? m : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (long k = 0; k < n_pix; ++k) {
            double T;
            int bd;
            long nf = composite_pixel(px[k] + 0.5, py[k] + 0.5, m, order, q, conic, opac, depth, depth_err, cfg,
                                      frags, &T, &bd, NULL);
            double C[3] = {0.0, 0.0, 0.0};
            for (long f = 0; f < nf; ++f) {
                long i = frags[f].i;
                for (int ch = 0; ch < 3; ++ch)
                    C[ch] += colour[3 * i + ch] * frags[f].alpha * frags[f].Tin;
            }
            for (int ch = 0; ch < 3; ++ch) rgb[3 * k + ch] = C[ch] + T * bg[ch];
            T_final[k] = T;
            n_contrib[k] = (int)nf;
            borderline[k] = (unsigned char)bd;
        }
        free(frags);
    }
    free(order);
    return 0;
}

/* One Gaussian's share of one pixel's gradient: dq_x, dq_y, dA, dB, dC,
 * dsigma, dc_r, dc_g, dc_b. */
typedef struct { long i; double a[9]; } orc_contrib;

/* A pixel's contributions and the Gaussians it flags as borderline. */
typedef struct { long n, nb; orc_contrib* c; long* b; } orc_pixel_out;

/* Backward of Eq. raster at one pixel centre (px, py) with dL/dI = g[3]:
 * fills out->c with one record per contributing Gaussian and out->b with the
 * Gaussians active at the pixel when it is borderline.
 * Written from the chain rule on Eq. raster: with T_k the transmittance in
 * front of fragment k and S_k the light composited behind it (including the
 * background through T_final),
 *   dI/dc_k = alpha_k T_k,  dI/dalpha_k = c_k T_k - S_k / (1 - alpha_k),
 * alpha_k = sigma_k G_k (unless clamped), G = exp(power),
 * power = -1/2 (A dx^2 + 2 B dx dy + C dy^2), dx = px - q_x.
 * A pixel with dL/dI = 0 contributes nothing to any gradient, so it is
 * skipped and flags nothing: its threshold decisions cannot change a
 * gradient. */
static void backward_pixel(double px, double py, const double* g, long m, const long* order,
                           const double* q, const double* conic, const double* opac,
                           const double* colour, const double* depth, const double* depth_err,
                           const double* cfg, orc_frag* frags, double* S, orc_pixel_out* out) {
    const double* bg = cfg + 5;
    double amax = cfg[1], amin = cfg[0];
    double T;
    int bd;
    long ncons;
    out->n = 0; out->nb = 0; out->c = NULL; out->b = NULL;
    if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) return;
    long nf = composite_pixel(px, py, m, order, q, conic, opac, depth, depth_err, cfg, frags, &T, &bd, &ncons);
    if (bd) {
        /* Every Gaussian that could be active here is unreliable. */
        out->b = (long*)malloc(sizeof(long) * (ncons > 0 ? ncons : 1));
        for (long k = 0; k < ncons && k < m; ++k) {
            long i = order[k];
            double dx = px - q[2 * i], dy = py - q[2 * i + 1];
            double pw = -0.5 * (conic[3 * i] * dx * dx + 2.0 * conic[3 * i + 1] * dx * dy +
                                conic[3 * i + 2] * dy * dy);
            if (opac[i] * exp(pw) >= amin * (1.0 - REL_BORDER)) out->b[out->nb++] = i;
        }
    }
    /* S_k = sum_{j>k} c_j alpha_j T_j + T_final bg, from the back. */
    double run[3] = {T * bg[0], T * bg[1], T * bg[2]};
    for (long f = nf - 1; f >= 0; --f) {
        for (int ch = 0; ch < 3; ++ch) S[3 * f + ch] = run[ch];
        long i = frags[f].i;
        for (int ch = 0; ch < 3; ++ch) run[ch] += colour[3 * i + ch] * frags[f].alpha * frags[f].Tin;
    }
    out->c = (orc_contrib*)calloc(nf > 0 ? nf : 1, sizeof(orc_contrib));
    out->n = nf;
    for (long f = 0; f < nf; ++f) {
        long i = frags[f].i;
        double* a = out->c[f].a;
        out->c[f].i = i;
        double al = frags[f].alpha, Tk = frags[f].Tin;
        double dLda = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            a[6 + ch] = al * Tk * g[ch];
            dLda += g[ch] * (colour[3 * i + ch] * Tk - S[3 * f + ch] / (1.0 - al));
        }
        if (frags[f].araw < amax) {
            double G = frags[f].G, sg = opac[i];
            double dx = frags[f].dx, dy = frags[f].dy;
            double A = conic[3 * i], B = conic[3 * i + 1], C = conic[3 * i + 2];
            double dLdpow = dLda * sg * G;
            a[5] = dLda * G;
            a[0] = dLdpow * (A * dx + B * dy);
            a[1] = dLdpow * (B * dx + C * dy);
            a[2] = dLdpow * (-0.5 * dx * dx);
            a[3] = dLdpow * (-dx * dy);
            a[4] = dLdpow * (-0.5 * dy * dy);
        }
    }
}

/* Gradient of the loss with respect to the per-Gaussian 2D quantities of one
 * view, over the pixels listed in (px, py) (n_pix >= 0) or, when px is NULL,
 * over every pixel of the W x H image.  dL_drgb is [3, H, W] for the full
 * image and [n_pix, 3] for a pixel list.  Outputs (accumulated, [n, k]):
 *   g_q [n,2]      dL/dq (pixel-space mean)
 *   g_conic [n,3]  dL/d(A, B, C) where the exponent is
 *                  -1/2 (A dx^2 + 2 B dx dy + C dy^2)
 *   g_opac [n]     dL/dsigma
 *   g_colour [n,3] dL/dc
 *   g_border [n]   set to 1 for Gaussians active at a borderline pixel.
 * Pixels are processed in parallel; their contributions are then added in
 * pixel order, so the result does not depend on the thread count. */
static int render_backward_impl(int W, int H, long n_pix, const int* pxs, const int* pys, long n,
                                const int* valid, const double* q, const double* conic,
                                const double* opac, const double* colour, const double* depth,
                                const double* depth_err, const double* cfg, const double* dL_drgb,
                                double* g_q,
                                double* g_conic, double* g_opac, double* g_colour,
                                unsigned char* g_border, int n_threads) {
    long* order = (long*)malloc(sizeof(long) * (n > 0 ? n : 1));
    long m = depth_order(n, valid, depth, order);
    int nthr = orc_threads(n_threads);
    (void)nthr;
    long total = pxs ? n_pix : (long)W * H;
    orc_pixel_out* outs = (orc_pixel_out*)calloc(total > 0 ? total : 1, sizeof(orc_pixel_out));
#ifdef _OPENMP
#pragma omp parallel num_threads(nthr)
#endif
    {
        orc_frag* frags = (orc_frag*)malloc(sizeof(orc_frag) * (m > 0 ? m : 1));
        double* S = (double*)malloc(sizeof(double) * 3 * (m > 0 ? m : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (long k = 0; k < total; ++k) {
            double px, py, g[3];
            if (pxs) {
                px = pxs[k] + 0.5; py = pys[k] + 0.5;
                for (int ch = 0; ch < 3; ++ch) g[ch] = dL_drgb[3 * k + ch];
            } else {
                px = (double)(k % W) + 0.5; py = (double)(k / W) + 0.5;
                for (int ch = 0; ch < 3; ++ch) g[ch] = dL_drgb[(long)ch * W * H + k];
            }
            backward_pixel(px, py, g, m, order, q, conic, opac, colour, depth, depth_err, cfg, frags, S,
                           &outs[k]);
        }
        free(S);
        free(frags);
    }
    for (long k = 0; k < total; ++k) {
        for (long f = 0; f < outs[k].n; ++f) {
            long i = outs[k].c[f].i;
            const double* a = outs[k].c[f].a;
            g_q[2 * i] += a[0]; g_q[2 * i + 1] += a[1];
            for (int c = 0; c < 3; ++c) g_conic[3 * i + c] += a[2 + c];
            g_opac[i] += a[5];
            for (int c = 0; c < 3; ++c) g_colour[3 * i + c] += a[6 + c];
        }
        for (long f = 0; f < outs[k].nb; ++f) g_border[outs[k].b[f]] = 1;
        free(outs[k].c);
        free(outs[k].b);
    }
    free(outs);
    free(order);
    return 0;
}

int orc_render_backward(int W, int H, long n, const int* valid, const double* q,
                        const double* conic, const double* opac, const double* colour,
                        const double* depth, const double* depth_err, const double* cfg,
                        const double* dL_drgb, double* g_q, double* g_conic, double* g_opac,
                        double* g_colour, unsigned char* g_border, int n_threads) {
    return render_backward_impl(W, H, 0, NULL, NULL, n, valid, q, conic, opac, colour, depth,
                                depth_err, cfg, dL_drgb, g_q, g_conic, g_opac, g_colour, g_border,
                                n_threads);
}

int orc_render_backward_pixels(long n_pix, const int* px, const int* py, long n, const int* valid,
                               const double* q, const double* conic, const double* opac,
                               const double* colour, const double* depth, const double* depth_err,
                               const double* cfg, const double* dL_drgb, double* g_q,
                               double* g_conic, double* g_opac, double* g_colour,
                               unsigned char* g_border, int n_threads) {
    return render_backward_impl(0, 0, n_pix, px, py, n, valid, q, conic, opac, colour, depth,
                                depth_err, cfg, dL_drgb, g_q, g_conic, g_opac, g_colour, g_border,
                                n_threads);
}

/* ---------- projection backward and pose gradient ---------- */

/* Chains dL/d(q, conic, sigma, colour) of one view back to the Gaussian
 * parameters (accumulated into g_*) and to the camera pose (accumulated
 * into g_pose[6] = dL/d(dphi, dt) for the left perturbation
 * T_CW <- Exp(dphi, dt) T_CW of the Appendix perturbation model).
 * g_border_colour is set to 1 where a colour channel sits within REL_BORDER of
 * its clamp. */
int orc_project_backward(long n, const double* means, const double* log_scales,
                         const double* quats, const double* opacity, const double* sh,
                         int sh_degree, const double* cam, const double* cfg,
                         const double* g_q, const double* g_conic, const double* g_opac,
                         const double* g_colour, double* g_means, double* g_log_scales,
                         double* g_quats, double* g_opacity, double* g_sh, double* g_pose,
                         unsigned char* g_border_colour) {
    int K = (sh_degree + 1) * (sh_degree + 1);
    const double* W = cam;
    double fx = cam[12], fy = cam[13];
    /* Gaussians are independent except for the pose gradient: each writes its
     * own pose term, and the terms are added in Gaussian order afterwards. */
    double* pose_i = g_pose ? (double*)calloc((size_t)(n > 0 ? n : 1) * 6, sizeof(double)) : NULL;
    int nthr = orc_threads(0);
    (void)nthr;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthr)
#endif
    for (long i = 0; i < n; ++i) {
        orc_proj P;
        const double* shi = sh + 3 * K * i;
        project_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, opacity[i], shi, sh_degree,
                    cam, cfg, &P);
        if (!P.valid) continue;
        double gmu[3] = {0, 0, 0}, gp[3] = {0, 0, 0};

        /* Colour: c = max(0, raw). */
        double graw[3];
        for (int ch = 0; ch < 3; ++ch) {
            graw[ch] = P.raw[ch] > 0.0 ? g_colour[3 * i + ch] : 0.0;
            if (fabs(P.raw[ch]) <= REL_BORDER) g_border_colour[i] = 1;
        }
        double Y[16], dY[16][3];
        sh_basis(P.dir, sh_degree, Y, dY);
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) g_sh[3 * K * i + 3 * k + ch] += Y[k] * graw[ch];
        double gd[3] = {0, 0, 0};
        if (sh_degree >= 1) {
            double gdir[3] = {0, 0, 0};
            for (int k = 1; k < K; ++k)
                for (int ch = 0; ch < 3; ++ch)
                    for (int c = 0; c < 3; ++c) gdir[c] += dY[k][c] * shi[3 * k + ch] * graw[ch];
            /* dir = d / |d|: g_d = (g_dir - dir (dir . g_dir)) / |d|. */
            double dotv = P.dir[0] * gdir[0] + P.dir[1] * gdir[1] + P.dir[2] * gdir[2];
            for (int k = 0; k < 3; ++k) gd[k] = (gdir[k] - P.dir[k] * dotv) / P.dlen;
            for (int k = 0; k < 3; ++k) gmu[k] += gd[k];
        }

        /* Opacity: sigma = 1 / (1 + exp(-o)). */
        g_opacity[i] += g_opac[i] * P.sigma * (1.0 - P.sigma);

        /* Conic = Sigma2^-1.  With G = [[gA, gB/2], [gB/2, gC]] the gradient as
         * a symmetric matrix, dL/dSigma2 = -Q G Q. */
        double Q[4] = {P.conic[0], P.conic[1], P.conic[1], P.conic[2]};
        double Gm[4] = {g_conic[3 * i], 0.5 * g_conic[3 * i + 1], 0.5 * g_conic[3 * i + 1],
                        g_conic[3 * i + 2]};
        double QG[4], G2[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) QG[2 * r + c] = Q[2 * r] * Gm[c] + Q[2 * r + 1] * Gm[2 + c];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) G2[2 * r + c] = -(QG[2 * r] * Q[c] + QG[2 * r + 1] * Q[2 + c]);

        /* Sigma2 = T Sigma3 T^T: dL/dSigma3 = T^T G2 T, dL/dT = 2 G2 T Sigma3. */
        double G3[9], gT[6];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int r = 0; r < 2; ++r)
                    for (int c = 0; c < 2; ++c) s += P.T[3 * r + a] * G2[2 * r + c] * P.T[3 * c + b];
                G3[3 * a + b] = s;
            }
        for (int r = 0; r < 2; ++r)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int k = 0; k < 3; ++k) s += G2[2 * r + c] * P.T[3 * c + k] * P.S3[3 * k + b];
                gT[3 * r + b] = 2.0 * s;
            }
        /* T = J W: dL/dJ = dL/dT W^T, dL/dW = J^T dL/dT. */
        double gJ[6], gW[9];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k) {
                double s = 0.0;
                for (int c = 0; c < 3; ++c) s += gT[3 * r + c] * W[3 * k + c];
                gJ[3 * r + k] = s;
            }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) gW[3 * a + b] = P.J[a] * gT[b] + P.J[3 + a] * gT[3 + b];

        /* J(p_C) and q(p_C). */
        double x = P.pc[0], y = P.pc[1], z = P.pc[2];
        double z2 = z * z, z3 = z2 * z;
        gp[0] += gJ[2] * (-fx / z2);
        gp[1] += gJ[5] * (-fy / z2);
        gp[2] += gJ[0] * (-fx / z2) + gJ[2] * (2.0 * fx * x / z3) + gJ[4] * (-fy / z2) +
                 gJ[5] * (2.0 * fy * y / z3);
        double gqx = g_q[2 * i], gqy = g_q[2 * i + 1];
        gp[0] += gqx * fx / z;
        gp[1] += gqy * fy / z;
        gp[2] += -gqx * fx * x / z2 - gqy * fy * y / z2;

        /* p_C = W mu + t. */
        for (int k = 0; k < 3; ++k) gmu[k] += W[k] * gp[0] + W[3 + k] * gp[1] + W[6 + k] * gp[2];

        /* Sigma3 = M M^T: dL/dM = 2 G3 M; M = R S. */
        double gM[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += G3[3 * a + k] * P.M[3 * k + b];
                gM[3 * a + b] = 2.0 * s;
            }
        double gR[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) gR[3 * a + b] = gM[3 * a + b] * P.sc[b];
        for (int b = 0; b < 3; ++b) {
            double gS = 0.0;
            for (int a = 0; a < 3; ++a) gS += gM[3 * a + b] * P.R[3 * a + b];
            g_log_scales[3 * i + b] += gS * P.sc[b];
        }
        /* R(qh): partial derivatives of each entry of the textbook formula. */
        double w = P.qh[0], qx = P.qh[1], qy = P.qh[2], qz = P.qh[3];
        double gqh[4] = {0, 0, 0, 0};
        gqh[0] = gR[1] * (-2 * qz) + gR[2] * (2 * qy) + gR[3] * (2 * qz) + gR[5] * (-2 * qx) +
                 gR[6] * (-2 * qy) + gR[7] * (2 * qx);
        gqh[1] = gR[1] * (2 * qy) + gR[2] * (2 * qz) + gR[3] * (2 * qy) + gR[4] * (-4 * qx) +
                 gR[5] * (-2 * w) + gR[6] * (2 * qz) + gR[7] * (2 * w) + gR[8] * (-4 * qx);
        gqh[2] = gR[0] * (-4 * qy) + gR[1] * (2 * qx) + gR[2] * (2 * w) + gR[3] * (2 * qx) +
                 gR[5] * (2 * qz) + gR[6] * (-2 * w) + gR[7] * (2 * qz) + gR[8] * (-4 * qy);
        gqh[3] = gR[0] * (-4 * qz) + gR[1] * (-2 * w) + gR[2] * (2 * qx) + gR[3] * (2 * w) +
                 gR[4] * (-4 * qz) + gR[5] * (2 * qy) + gR[6] * (2 * qx) + gR[7] * (2 * qy);
        /* qh = quat / |quat|. */
        double dq = gqh[0] * P.qh[0] + gqh[1] * P.qh[1] + gqh[2] * P.qh[2] + gqh[3] * P.qh[3];
        for (int k = 0; k < 4; ++k) g_quats[4 * i + k] += (gqh[k] - P.qh[k] * dq) / P.qn;

        for (int k = 0; k < 3; ++k) g_means[3 * i + k] += gmu[k];

        /* Pose, left perturbation: p_C <- p_C + dphi x p_C + dt, W <- W + [dphi]x W,
         * campos <- campos - W^T dt. */
        if (pose_i) {
            double gW_Wt[9];
            double* gpi = pose_i + 6 * i;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k) s += gW[3 * a + k] * W[3 * b + k];
                    gW_Wt[3 * a + b] = s;
                }
            gpi[0] = (P.pc[1] * gp[2] - P.pc[2] * gp[1]) + (gW_Wt[7] - gW_Wt[5]);
            gpi[1] = (P.pc[2] * gp[0] - P.pc[0] * gp[2]) + (gW_Wt[2] - gW_Wt[6]);
            gpi[2] = (P.pc[0] * gp[1] - P.pc[1] * gp[0]) + (gW_Wt[3] - gW_Wt[1]);
            for (int k = 0; k < 3; ++k)
                gpi[3 + k] = gp[k] + (W[3 * k] * gd[0] + W[3 * k + 1] * gd[1] + W[3 * k + 2] * gd[2]);
        }
    }
    if (pose_i) {
        for (long i = 0; i < n; ++i)
            for (int k = 0; k < 6; ++k) g_pose[k] += pose_i[6 * i + k];
        free(pose_i);
    }
    return 0;
}

/* ---------- pose Jacobian of the rendered pixels (Sec. II-D) ---------- */

/* Tangents of one Gaussian's projected quantities with respect to the
 * left-perturbed camera pose xi = [dphi; dt], T_CW <- Exp(xi) T_CW (Appendix
 * A, perturbation model), written forward from Eqs. q and spat:
 *   dp_C/ddphi_k = e_k x p_C,   dp_C/ddt_k = e_k,
 *   dW/ddphi_k = [e_k]x W,      campos = -W^T t moves by -W^T dt only,
 *   q = pi(p_C):  dq = J dp_C,
 *   T = J W:      dT = dJ W + J dW with dJ from J(p_C),
 *   Sigma2 = T Sigma3 T^T + b I:  dSigma2 = dT Sigma3 T^T + T Sigma3 dT^T,
 *   conic = Sigma2^-1:            dconic = -conic dSigma2 conic,
 *   colour = max(0, SH(dir)), dir = (mu - campos) / |mu - campos|.
 * Outputs (column k = d/dxi_k): dq[2][6], dconic[3][6] (A, B, C) and
 * dcol[3][6]. */
static void pose_tangents(const orc_proj* P, const double* cam, const double* sh, int sh_degree,
                          double dq[2][6], double dconic[3][6], double dcol[3][6]) {
    const double* W = cam;
    double fx = cam[12], fy = cam[13];
    double x = P->pc[0], y = P->pc[1], z = P->pc[2];
    for (int k = 0; k < 6; ++k) {
        /* dp_C and dW for xi = e_k */
        double dp[3] = {0, 0, 0}, dW[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (k < 3) {
            double e[3] = {0, 0, 0};
            e[k] = 1.0;
            dp[0] = e[1] * z - e[2] * y;
            dp[1] = e[2] * x - e[0] * z;
            dp[2] = e[0] * y - e[1] * x;
            /* [e]x W: row r of [e]x is (e x .) applied to the columns of W */
            for (int c = 0; c < 3; ++c) {
                double w0 = W[c], w1 = W[3 + c], w2 = W[6 + c];
                dW[c] = e[1] * w2 - e[2] * w1;
                dW[3 + c] = e[2] * w0 - e[0] * w2;
                dW[6 + c] = e[0] * w1 - e[1] * w0;
            }
        } else {
            dp[k - 3] = 1.0;
        }
        /* q = (fx x / z + cx, fy y / z + cy) */
        dq[0][k] = P->J[0] * dp[0] + P->J[1] * dp[1] + P->J[2] * dp[2];
        dq[1][k] = P->J[3] * dp[0] + P->J[4] * dp[1] + P->J[5] * dp[2];
        /* J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]] */
        double dJ[6];
        dJ[0] = -fx * dp[2] / (z * z);
        dJ[1] = 0.0;
        dJ[2] = -fx * dp[0] / (z * z) + 2.0 * fx * x * dp[2] / (z * z * z);
        dJ[3] = 0.0;
        dJ[4] = -fy * dp[2] / (z * z);
        dJ[5] = -fy * dp[1] / (z * z) + 2.0 * fy * y * dp[2] / (z * z * z);
        double dT[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int m = 0; m < 3; ++m) s += dJ[3 * r + m] * W[3 * m + c] + P->J[3 * r + m] * dW[3 * m + c];
                dT[3 * r + c] = s;
            }
        /* dSigma2 = dT S3 T^T + T S3 dT^T */
        double dS[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) {
                double s = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        s += dT[3 * r + i] * P->S3[3 * i + j] * P->T[3 * c + j] +
                             P->T[3 * r + i] * P->S3[3 * i + j] * dT[3 * c + j];
                dS[2 * r + c] = s;
            }
        double Q[4] = {P->conic[0], P->conic[1], P->conic[1], P->conic[2]};
        double QdS[4], dQ[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) QdS[2 * r + c] = Q[2 * r] * dS[c] + Q[2 * r + 1] * dS[2 + c];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) dQ[2 * r + c] = -(QdS[2 * r] * Q[c] + QdS[2 * r + 1] * Q[2 + c]);
        dconic[0][k] = dQ[0];
        dconic[1][k] = 0.5 * (dQ[1] + dQ[2]);
        dconic[2][k] = dQ[3];
        /* colour: dvec = mu - campos, d campos/d dt_j = -W^T e_j = -(row j of W) */
        double ddv[3] = {0, 0, 0};
        if (k >= 3)
            for (int i = 0; i < 3; ++i) ddv[i] = W[3 * (k - 3) + i];
        double dd = P->dir[0] * ddv[0] + P->dir[1] * ddv[1] + P->dir[2] * ddv[2];
        double ddir[3];
        for (int i = 0; i < 3; ++i) ddir[i] = (ddv[i] - P->dir[i] * dd) / P->dlen;
        double Y[16], dY[16][3];
        int K = (sh_degree + 1) * (sh_degree + 1);
        sh_basis(P->dir, sh_degree, Y, dY);
        for (int ch = 0; ch < 3; ++ch) {
            double draw = 0.0;
            for (int m = 1; m < K; ++m)
                draw += (dY[m][0] * ddir[0] + dY[m][1] * ddir[1] + dY[m][2] * ddir[2]) * sh[3 * m + ch];
            dcol[ch][k] = P->raw[ch] > 0.0 ? draw : 0.0;
        }
    }
}

/* Per-pixel pose Jacobian of the rendered colour, H[p][ch][k] = dI_ch(x_p) /
 * dxi_k, by forward-mode differentiation of Eq. raster at the listed pixels
 * of one view (the measurement Jacobian of the photometric update, Sec. II-D,
 * Eq. minimization).  With T_j the transmittance in front of fragment j,
 *   I = sum_j c_j alpha_j T_j + T_final bg,  T_{j+1} = T_j (1 - alpha_j),
 *   dI = sum_j (dc_j alpha_j T_j + c_j dalpha_j T_j + c_j alpha_j dT_j)
 *        + dT_final bg,  dT_{j+1} = dT_j (1 - alpha_j) - T_j dalpha_j,
 *   alpha_j = sigma_j G_j (0 derivative where clamped), G = exp(power),
 *   dpower = -1/2 (dA dx^2 + 2 dB dx dy + dC dy^2)
 *            + (A dx + B dy) dq_x + (B dx + C dy) dq_y.
 * The fragment list (which Gaussians contribute, in which order) is the one
 * composite_pixel decides; culling is locally constant.  rgb [n_pix][3] and
 * borderline [n_pix] as orc_render_pixels. */
int orc_pose_jacobian_pixels(long n_pix, const int* pxs, const int* pys, long n, const double* means,
                             const double* log_scales, const double* quats, const double* opacity,
                             const double* sh, int sh_degree, const double* cam, const double* cfg,
                             double* Hout, double* rgb, unsigned char* borderline, int n_threads) {
    int K = (sh_degree + 1) * (sh_degree + 1);
    const double* bg = cfg + 5;
    double amax = cfg[1];
    orc_proj* P = (orc_proj*)malloc(sizeof(orc_proj) * (n > 0 ? n : 1));
    int* valid = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    double* q = (double*)malloc(sizeof(double) * 2 * (n > 0 ? n : 1));
    double* conic = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double* opac = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
    double* depth = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
    double* zerr = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
    double* tq = (double*)malloc(sizeof(double) * 12 * (n > 0 ? n : 1));
    double* tc = (double*)malloc(sizeof(double) * 18 * (n > 0 ? n : 1));
    double* tcol = (double*)malloc(sizeof(double) * 18 * (n > 0 ? n : 1));
    long* order = (long*)malloc(sizeof(long) * (n > 0 ? n : 1));
    for (long i = 0; i < n; ++i) {
        project_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, opacity[i], sh + 3 * K * i, sh_degree,
                    cam, cfg, &P[i]);
        valid[i] = P[i].valid;
        q[2 * i] = P[i].q[0];
        q[2 * i + 1] = P[i].q[1];
        for (int k = 0; k < 3; ++k) conic[3 * i + k] = P[i].conic[k];
        opac[i] = P[i].sigma;
        depth[i] = P[i].pc[2];
        zerr[i] = P[i].zerr;
        if (P[i].valid) {
            double dq[2][6], dcn[3][6], dcol[3][6];
            pose_tangents(&P[i], cam, sh + 3 * K * i, sh_degree, dq, dcn, dcol);
            memcpy(tq + 12 * i, dq, sizeof(dq));
            memcpy(tc + 18 * i, dcn, sizeof(dcn));
            memcpy(tcol + 18 * i, dcol, sizeof(dcol));
        }
    }
    long m = depth_order(n, valid, depth, order);
    int nthr = orc_threads(n_threads);
    (void)nthr;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthr)
#endif
    {
        orc_frag* frags = (orc_frag*)malloc(sizeof(orc_frag) * (m > 0 ? m : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (long p = 0; p < n_pix; ++p) {
            double T;
            int bd;
            long nf = composite_pixel(pxs[p] + 0.5, pys[p] + 0.5, m, order, q, conic, opac, depth, zerr, cfg,
                                      frags, &T, &bd, NULL);
            double C[3] = {0, 0, 0}, dC[3][6], dT[6];
            memset(dC, 0, sizeof(dC));
            memset(dT, 0, sizeof(dT));
            for (long f = 0; f < nf; ++f) {
                long i = frags[f].i;
                double dx = frags[f].dx, dy = frags[f].dy, a = frags[f].alpha, Tj = frags[f].Tin;
                double A = conic[3 * i], B = conic[3 * i + 1], Cc = conic[3 * i + 2];
                const double* dq = tq + 12 * i;     /* [2][6] */
                const double* dcn = tc + 18 * i;    /* [3][6] */
                const double* dcol = tcol + 18 * i; /* [3][6] */
                double da[6];
                for (int k = 0; k < 6; ++k) {
                    double dpow = -0.5 * (dcn[k] * dx * dx + 2.0 * dcn[6 + k] * dx * dy + dcn[12 + k] * dy * dy) +
                                  (A * dx + B * dy) * dq[k] + (B * dx + Cc * dy) * dq[6 + k];
                    da[k] = frags[f].araw < amax ? a * dpow : 0.0;
                }
                for (int ch = 0; ch < 3; ++ch) {
                    double c = P[i].colour[ch];
                    C[ch] += c * a * Tj;
                    for (int k = 0; k < 6; ++k)
                        dC[ch][k] += dcol[6 * ch + k] * a * Tj + c * da[k] * Tj + c * a * dT[k];
                }
                for (int k = 0; k < 6; ++k) dT[k] = dT[k] * (1.0 - a) - Tj * da[k];
            }
            for (int ch = 0; ch < 3; ++ch) {
                rgb[3 * p + ch] = C[ch] + T * bg[ch];
                for (int k = 0; k < 6; ++k) Hout[18 * p + 6 * ch + k] = dC[ch][k] + dT[k] * bg[ch];
            }
            borderline[p] = (unsigned char)bd;
        }
        free(frags);
    }
    free(P); free(valid); free(q); free(conic); free(opac); free(depth); free(zerr);
    free(tq); free(tc); free(tcol); free(order);
    return 0;
}

/* ---------- Adam (Sec. II-B.2) ---------- */

/* Kingma & Ba (2015) with bias correction, in the form torch.optim.Adam uses:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr / (1 - b1^t) * m / (sqrt(v) / sqrt(1 - b2^t) + eps). */
void orc_adam(long n, double* p, const double* g, double* m, double* v, double lr, double b1,
              double b2, double eps, long step) {
    double bc1 = 1.0 - pow(b1, (double)step);
    double bc2 = 1.0 - pow(b2, (double)step);
    for (long i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double denom = sqrt(v[i]) / sqrt(bc2) + eps;
        p[i] -= (lr / bc1) * m[i] / denom;
    }
}

int orc_num_threads(void) { return orc_threads(0); }
