"""Write dd_log_table.cuh: the tables of the table-driven double logarithm of
dd_common.cuh (Tang, "Table-driven implementation of the logarithm function in
IEEE floating-point arithmetic", ACM TOMS 16, 1990): for c_j = 1 + j/128,
j = -32..64 (the reduced argument lies in [0.75, 1.5)), log(c_j) and 1/c_j
rounded to double, as exact hexadecimal literals, at index j + 32.
Run: python gen_log_table.py > dd_log_table.cuh"""
import math


def main():
    js = range(-32, 65)
    logs = [math.log(1.0 + j / 128.0) for j in js]
    invs = [1.0 / (1.0 + j / 128.0) for j in js]
    print("// Generated by gen_log_table.py: log(1 + j/128) and 1/(1 + j/128) at index j + 32, j = -32..64,")
    print("// rounded to double.")
    print("#pragma once")
    for name, vals in (("kLogC", logs), ("kInvC", invs)):
        print(f"static __device__ const double {name}[97] = {{")
        for j in range(0, 97, 3):
            print("    " + ", ".join(float.hex(v) for v in vals[j:j + 3]) + ",")
        print("};")


if __name__ == "__main__":
    main()
