"""Write log_table.cuh: the tables of the FP64 logarithm in fmath64.cuh (Tang's table-driven method,
ACM TOMS 16(4), 1990).  For F_j = 1 + j/128, j = 0..128: ln F_j split into a lead that is a multiple
of 2^-42 (so that k ln2_lead + lead_j is exact for every exponent k of a double) and a trail, and
1/F_j rounded to double.  ln 2 is split the same way.  Values from 60-digit decimal arithmetic.

    python gen_log_table.py > log_table.cuh
"""
from decimal import Decimal, getcontext

getcontext().prec = 60
SCALE = Decimal(2) ** 42


def split(v: Decimal):
    lead = (v * SCALE).to_integral_value() / SCALE
    return float(lead), float(v - lead)


def hexd(x: float) -> str:
    return float.hex(x)


def main():
    ln2 = Decimal(2).ln()
    l2h, l2t = split(ln2)
    rows = []
    for j in range(129):
        F = 1 + Decimal(j) / 128
        lh, lt = split(F.ln())
        rows.append((lh, lt, float(1 / F)))
    print("// Generated by gen_log_table.py (do not edit): Tang's logarithm tables, see fmath64.cuh.")
    print("#pragma once")
    print("#include \"fmath64_defs.cuh\"")
    print("namespace art {")
    print(f"constexpr double LOG_LN2_LEAD = {hexd(l2h)};")
    print(f"constexpr double LOG_LN2_TRAIL = {hexd(l2t)};")
    print("// {lead of ln F_j, trail of ln F_j, 1/F_j}, F_j = 1 + j/128")
    print("ART_FM_TABLE const double LOG_TABLE[129][3] = {")
    for lh, lt, inv in rows:
        print(f"    {{{hexd(lh)}, {hexd(lt)}, {hexd(inv)}}},")
    print("};")
    print("}  // namespace art")


if __name__ == "__main__":
    main()
