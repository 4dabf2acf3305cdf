"""Shares of the comparisons the parity tests leave out, collected so the
test run can print them.

A pixel is left out of an image comparison when the oracle flags one of its
threshold decisions as borderline (within 1e-5 relative of its cut, where
FP32 and FP64 may decide differently).  The loss gradient is zero at such
pixels on both sides, so no Gaussian is left out of a gradient comparison
for them; a Gaussian is left out only when one of its colour channels sits
within 1e-5 of the clamp at 0.
"""
import os

RECORDS = []
REPORTS = []


def record(kind, share, bound, count, total, allow=0):
    """One comparison: `count` of `total` left out, against a bound on the
    share plus `allow` items of count noise (the test asserts
    count <= bound * total + allow)."""
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    RECORDS.append((test, kind, float(share), float(bound), int(count), int(total), int(allow)))


def report(title, lines):
    """A table of measured errors to print with the summary."""
    REPORTS.append((title, list(lines)))


def report_lines():
    out = []
    for title, lines in REPORTS:
        out.append(title)
        out.extend("  " + ln for ln in lines)
    return out


def summary_lines():
    if not RECORDS:
        return []
    out = ["%-78s %-9s %10s %10s %10s" % ("test", "excluded", "share", "bound", "count/total")]
    worst = {}
    # per (test, kind): the comparison that used most of what it was allowed
    # (count / (bound * total + allow)), and the totals
    for test, kind, share, bound, count, total, allow in RECORDS:
        key = (test, kind)
        use = count / max(bound * total + allow, 1e-30)
        u, s, b, c0, t0, a, c, t = worst.get(key, (-1.0, 0.0, bound, 0, 0, allow, 0, 0))
        if use > u:
            u, s, b, c0, t0, a = use, share, bound, count, total, allow
        worst[key] = (u, s, b, c0, t0, a, c + count, t + total)
    for (test, kind), (u, s, b, c0, t0, a, c, t) in worst.items():
        out.append("%-78s %-9s %10.2e %10.2e %5d/%d" % (test[-78:], kind, s, b, c, t))
    for kind in sorted({k for _, k in worst}):
        rows = [(v[0], v, test) for (test, k), v in worst.items() if k == kind]
        _, (u, s, b, c0, t0, a, _c, _t), test = max(rows, key=lambda r: r[0])
        tot_c = sum(v[6] for (test_, k), v in worst.items() if k == kind)
        tot_t = sum(v[7] for (test_, k), v in worst.items() if k == kind)
        noise = " plus %d of count noise" % a if a else ""
        out.append("%s excluded: %d of %d (%.2e) over %d comparisons; closest to its limit: %d of %d (share %.2e) "
                   "against a bound of %.2e%s in %s (%.0f %% of the allowed count)"
                   % (kind, tot_c, tot_t, tot_c / max(tot_t, 1), len(rows), c0, t0, s, b, noise,
                      test.split("::")[-1], 100.0 * u))
    return out
