"""Writes csrc/exp2q_table.h: EXP2Q[f] = round(2^(23 - f/256)), f = 0..255, the table of the
integer softmax that turns the context model's logits into 16-bit frequencies.

Computed with Python's decimal module at 50 significant digits, 2^x = exp(x ln 2), then
rounded to the nearest integer (no entry lies within 1e-30 of a half-integer).  Run it to
regenerate the header; the committed header is what the library compiles."""
from __future__ import annotations

import decimal
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def table() -> list[int]:
    ctx = decimal.Context(prec=50)
    ln2 = ctx.ln(decimal.Decimal(2))
    out = []
    for f in range(256):
        x = ctx.multiply(ctx.subtract(decimal.Decimal(23), ctx.divide(decimal.Decimal(f), decimal.Decimal(256))), ln2)
        y = ctx.exp(x)
        r = int(y.to_integral_value(rounding=decimal.ROUND_HALF_UP))
        assert abs(y - r) < decimal.Decimal("0.5") - decimal.Decimal("1e-30")
        out.append(r)
    return out


def write(path: str = os.path.join(HERE, "csrc", "exp2q_table.h")) -> None:
    t = table()
    lines = ["// Generated by gen_exp2q.py: EXP2Q[f] = round(2^(23 - f/256)), f = 0..255.",
             "#pragma once", "#define SGS_EXP2Q_VALUES \\"]
    for i in range(0, 256, 8):
        sep = ", \\" if i + 8 < 256 else ""
        lines.append("    " + ", ".join("%du" % v for v in t[i:i + 8]) + sep)
    lines += [""]
    open(path, "w").write("\n".join(lines))


if __name__ == "__main__":
    write()
