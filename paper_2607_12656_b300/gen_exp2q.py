"""Writes csrc/exp2q_table.h: EXP2Q[f] = round(2^(23 - f/256)), f = 0..255, the table of the
integer softmax that turns the context model's logits into 16-bit frequencies, and
csrc/sin8_table.h: the 8-bit sine table of the Fourier positional embedding.

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


def sin8() -> list[int]:
    """SIN8[j] = round(127 sin(2 pi j / 256)), j = 0..255: the phase table of the Fourier
    positional embedding.  sin by its Taylor series at 50 significant digits (pi from
    Machin's formula), then rounded to the nearest integer (no entry lies within 1e-6 of a
    half-integer)."""
    ctx = decimal.Context(prec=50)
    D = decimal.Decimal

    def arctan_inv(x: int) -> decimal.Decimal:  # arctan(1/x) by its series
        total, term, k = D(0), ctx.divide(D(1), D(x)), 0
        x2 = D(x * x)
        while term != 0:
            total = ctx.add(total, ctx.divide(term, D(2 * k + 1)) if k % 2 == 0 else -ctx.divide(term, D(2 * k + 1)))
            term = ctx.divide(term, x2)
            k += 1
        return total

    pi = ctx.multiply(D(4), ctx.subtract(ctx.multiply(D(4), arctan_inv(5)), arctan_inv(239)))
    out = []
    for j in range(256):
        x = ctx.divide(ctx.multiply(ctx.multiply(D(2), pi), D(j)), D(256))
        x = ctx.subtract(x, ctx.multiply(D(2), pi)) if j >= 128 else x  # |x| <= pi
        total, term, k = D(0), x, 1
        while abs(term) > D("1e-45"):
            total = ctx.add(total, term)
            term = ctx.divide(ctx.multiply(ctx.multiply(term, x), x), D(-(k + 1) * (k + 2)))
            k += 2
        y = ctx.multiply(D(127), total)
        r = int(y.to_integral_value(rounding=decimal.ROUND_HALF_UP))
        assert abs(abs(y - r) - D("0.5")) > D("1e-6")
        out.append(r)
    return out


def write_sin8(path: str = os.path.join(HERE, "csrc", "sin8_table.h")) -> None:
    t = sin8()
    lines = ["// Generated by gen_exp2q.py: SIN8[j] = round(127 sin(2 pi j / 256)), j = 0..255.",
             "#pragma once", "#define SGS_SIN8_VALUES \\"]
    for i in range(0, 256, 16):
        sep = ", \\" if i + 16 < 256 else ""
        lines.append("    " + ", ".join("%d" % v for v in t[i:i + 16]) + sep)
    lines += [""]
    open(path, "w").write("\n".join(lines))


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
    write_sin8()
