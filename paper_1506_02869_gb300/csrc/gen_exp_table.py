"""Writes exp_table.h: the constants of the normalisation's FP64 exponential.

The table-driven method of Tang (ACM TOMS 15(2), 1989) needs 2^(j/256),
j = 0..255, and ln(2)/256 split into a head L1 (the double nearest to it) and
the tail L2 = ln(2)/256 - L1.  Every value is computed here with 60 decimal
digits and rounded once to the nearest double (Python's float(Decimal) is
correctly rounded).  Run: python gen_exp_table.py > exp_table.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 60
ln2 = Decimal(2).ln()
step = ln2 / 256
L1 = float(step)
L2 = float(step - Decimal(L1))
tab = [float(Decimal(2) ** (Decimal(j) / 256)) for j in range(256)]

print("// Generated by gen_exp_table.py (this directory): 2^(j/256) rounded to the")
print("// nearest double, and ln(2)/256 = kExpL1 + kExpL2 (head and tail).")
print("#pragma once")
print()
print("namespace tma {")
print()
print(f"constexpr double kExpL1 = {L1.hex()};  // {L1!r}")
print(f"constexpr double kExpL2 = {L2.hex()};  // {L2!r}")
print()
print("__device__ const double kExp2Frac[256] = {")
for i in range(0, 256, 2):
    print(f"    {tab[i].hex()}, {tab[i + 1].hex()},")
print("};")
print()
print("}  // namespace tma")
