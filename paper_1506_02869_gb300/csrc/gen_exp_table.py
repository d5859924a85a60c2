"""Writes exp_table.h: the constants of the normalisation's exponential.

The table-driven method of Tang (ACM TOMS 15(2), 1989), evaluated in integer
fixed point: exp(x) = 2^(k >> 8) 2^((k & 255)/256) exp(r), x = k ln2/256 + r.
It needs 2^(j/256), j = 0..255, as 64-bit integers at the scale 2^63 (each
rounded once to the nearest integer), and ln(2)/256 at the scale 2^53 split
into an integer head C1 and a tail C2 at a further 2^32 (rounded to the
nearest integer), so that k ln2/256 at the scale 2^53 is k C1 + (k C2) / 2^32.
Every value is computed here with 60 decimal digits.
Run: python gen_exp_table.py > exp_table.h
"""
from decimal import ROUND_HALF_EVEN, Decimal, getcontext

getcontext().prec = 60
ln2 = Decimal(2).ln()
step53 = ln2 / 256 * (Decimal(2) ** 53)
C1 = int(step53.to_integral_value(rounding=ROUND_HALF_EVEN))
C2 = int(((step53 - C1) * (Decimal(2) ** 32)).to_integral_value(rounding=ROUND_HALF_EVEN))
tab = [int((Decimal(2) ** (Decimal(j) / 256) * (Decimal(2) ** 63)).to_integral_value(rounding=ROUND_HALF_EVEN))
       for j in range(256)]

print("// Generated by gen_exp_table.py (this directory): 2^(j/256) at the scale 2^63")
print("// rounded to the nearest integer, and ln(2)/256 at the scale 2^53 as the")
print("// integer head kExpC1 plus the tail kExpC2 / 2^32.")
print("#pragma once")
print()
print("#include <stdint.h>")
print()
print("namespace tma {")
print()
print(f"constexpr long long kExpC1 = {C1}LL;")
print(f"constexpr long long kExpC2 = {C2}LL;")
print()
print("__device__ const unsigned long long kExp2Frac63[256] = {")
for i in range(0, 256, 4):
    print("    " + ", ".join(f"0x{tab[i + d]:016x}ull" for d in range(4)) + ",")
print("};")
print()
print("}  // namespace tma")
