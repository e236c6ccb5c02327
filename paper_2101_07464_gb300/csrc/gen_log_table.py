"""Writes hd_log_table.cuh: the table of the FP64 logarithm used by the Gaussian draws.

For i = -64 .. 128, entry i + 64 holds c_i = 1 / (1 + i / 256) rounded to an FP32 value
(stored as an FP64 value, exact) and T_i = -ln(c_i) rounded to the nearest FP64 value.  The
logarithm is evaluated with 40 significant decimal digits (Python's decimal module), so T_i is
correctly rounded.  For i = 0, c_0 = 1 and T_0 = 0 exactly.  Run from this directory:
python gen_log_table.py > hd_log_table.cuh
"""
import decimal
import struct
import sys


def f32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def main(out=sys.stdout):
    decimal.getcontext().prec = 40
    out.write("// Generated by gen_log_table.py: {c_i, -ln c_i} for i = -64 .. 128, c_i = fp32(1 / (1 + i/256)).\n")
    out.write("#pragma once\n\n")
    out.write("namespace hd {\n\n")
    out.write("constexpr int kLogTabLo = -64;\n")
    out.write("constexpr int kLogTabN = 193;\n")
    out.write("static __device__ const double2 kLogTab[kLogTabN] = {\n")
    for i in range(-64, 129):
        c = f32(1.0 / (1.0 + i / 256.0))
        t = -decimal.Decimal(c).ln() if i != 0 else decimal.Decimal(0)
        out.write("    {%s, %s},\n" % (float(c).hex(), float(t).hex()))
    out.write("};\n\n}  // namespace hd\n")


if __name__ == "__main__":
    main()
