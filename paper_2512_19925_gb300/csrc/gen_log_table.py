"""Writes log_table.inc, the reduction table of the device logarithm
(hw_log in hww_device.cuh): for j = 0..127 (the top 7 mantissa bits of
m in [1, 2)),

    j < 64:  c = 1 + j/128,           IC_j = 1/c rounded,       K_j = 0
    j >= 64: c = (1 + (j+1)/128) / 2, IC_j = (1/c rounded) / 2, K_j = 1
    T_j = -log(IC_j 2^K_j), rounded once to double.

IC_j is computed in IEEE double arithmetic (Python floats); T_j from the
decimal module at 60 digits, then rounded to the nearest double.  Run it
from this directory:  python gen_log_table.py
"""
import decimal
import os

decimal.getcontext().prec = 60


def table():
    rows = []
    for j in range(128):
        if j < 64:
            ic = 1.0 / (1.0 + j / 128.0)
            y = ic
        else:
            inv = 1.0 / ((1.0 + (j + 1) / 128.0) * 0.5)
            ic = inv * 0.5
            y = inv
        t = float(-decimal.Decimal(y).ln())
        rows.append((ic, t))
    return rows


def render(rows):
    lines = ["// Generated by gen_log_table.py: the reduction table of hw_log", "// (1/c_j rounded, halved for j >= 64; T_j = -log(IC_j 2^K_j) rounded).",
             "static __device__ const double LOG_IC[128] = {"]
    lines += ["    %s," % ic.hex() for ic, _ in rows]
    lines += ["};", "static __device__ const double LOG_T[128] = {"]
    lines += ["    %s," % t.hex() for _, t in rows]
    lines += ["};", ""]
    return "\n".join(lines)


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "log_table.inc"), "w") as f:
        f.write(render(table()))
