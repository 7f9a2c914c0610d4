"""Writes csrc/fft_twiddle_table.inc: w^n = exp(2 pi i n / 512), n = 0..511.

The table is evaluated in x87 extended precision (numpy longdouble) and rounded
once to double; a second table holds each value as a float pair (hi, lo) with
hi = fl32(x) and lo = fl32(x - hi), for the double-float transforms.  Values are
written as C99 hex floats so the compiled constants are bit-exact.  Run by the
build when the file is missing; the output is committed.
"""
import os

import numpy as np

MAXLEN = 512
_PI = np.longdouble("3.14159265358979323846264338327950288419716939937510")


def main(path=None):
    here = os.path.dirname(os.path.abspath(__file__))
    path = path or os.path.join(here, "csrc", "fft_twiddle_table.inc")
    n = np.arange(MAXLEN, dtype=np.longdouble)
    ang = 2 * _PI * n / np.longdouble(MAXLEN)
    c = np.cos(ang)
    s = np.sin(ang)
    cd = c.astype(np.float64)
    sd = s.astype(np.float64)
    lines = ["// generated by gen_twiddles.py: exp(2 pi i n / 512) as double2, then as float pairs"]
    lines.append("#define NSPT_TWIDDLE_D2 \\")
    for i in range(MAXLEN):
        sep = "," if i + 1 < MAXLEN else ""
        lines.append("  {%s, %s}%s \\" % (float(cd[i]).hex(), float(sd[i]).hex(), sep))
    lines.append("")
    ch = c.astype(np.float32)
    sh = s.astype(np.float32)
    cl = (c - ch.astype(np.longdouble)).astype(np.float32)
    sl = (s - sh.astype(np.longdouble)).astype(np.float32)
    lines.append("#define NSPT_TWIDDLE_F4 \\")
    for i in range(MAXLEN):
        sep = "," if i + 1 < MAXLEN else ""
        vals = [float(v).hex() for v in (ch[i], cl[i], sh[i], sl[i])]
        lines.append("  {%sf, %sf, %sf, %sf}%s \\" % (vals[0].replace("0x", "0x"), vals[1], vals[2], vals[3], sep))
    lines.append("")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return path


if __name__ == "__main__":
    print(main())
