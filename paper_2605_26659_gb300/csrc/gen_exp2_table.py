"""Write exp2_table.h: the 64 float64 values 2^(k/64), k = 0..63, of the
table-driven 2^x of the float64 kernels (P. T. P. Tang, "Table-driven
implementation of the exponential function in IEEE floating-point
arithmetic", ACM TOMS 15(2), 1989).

Each value is computed with Python's decimal module at 60 significant digits
and rounded once to the nearest float64 (float(Decimal) rounds correctly),
then written as an exact hexadecimal literal.  Run from this directory:
    python gen_exp2_table.py > exp2_table.h
"""
from decimal import Decimal, getcontext


def table():
    getcontext().prec = 60
    ln2 = Decimal(2).ln()
    return [float((ln2 * k / 64).exp()) for k in range(64)]


def main():
    vals = table()
    print("// 2^(k/64), k = 0..63, each the float64 nearest to the exact value;")
    print("// written by gen_exp2_table.py (decimal arithmetic, 60 digits).")
    print("#pragma once")
    print()
    print("namespace finom {")
    print("namespace {")
    print("__device__ const double kExp2Tab[64] = {")
    for i in range(0, 64, 2):
        print(f"    {vals[i].hex()}, {vals[i + 1].hex()},")
    print("};")
    print("}  // namespace")
    print("}  // namespace finom")


if __name__ == "__main__":
    main()
