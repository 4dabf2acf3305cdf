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


def record(kind, share, bound, count, total):
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    RECORDS.append((test, kind, float(share), float(bound), int(count), int(total)))


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
    for test, kind, share, bound, count, total in RECORDS:
        key = (test, kind)
        s, b, c, t = worst.get(key, (0.0, bound, 0, 0))
        worst[key] = (max(s, share), bound if share >= s else b, c + count, t + total)
    for (test, kind), (s, b, c, t) in worst.items():
        out.append("%-78s %-9s %10.2e %10.2e %5d/%d" % (test[-78:], kind, s, b, c, t))
    for kind in sorted({k for _, k in worst}):
        rows = [(s / b if b > 0 else 0.0, s, b, test) for (test, k), (s, b, c, t) in worst.items() if k == kind]
        r, s, b, test = max(rows)
        tot_c = sum(c for (test_, k), (s_, b_, c, t) in worst.items() if k == kind)
        tot_t = sum(t for (test_, k), (s_, b_, c, t) in worst.items() if k == kind)
        out.append("%s excluded: %d of %d (%.2e) over %d comparisons; largest share %.2e against its bound "
                   "%.2e in %s" % (kind, tot_c, tot_t, tot_c / max(tot_t, 1), len(rows), s, b, test.split("::")[-1]))
    return out
