"""Writes dp5_nystrom.h: Dormand-Prince 5(4) coefficients rearranged for a second-order system.

For y = (x, v) with x' = v and v' = a(t, x) (the force does not depend on velocities), the stage
velocities of an explicit Runge-Kutta method never need to be formed: stage s has
    x_s = x + c_s h v + h^2 sum_m (A A)_{sm} a_m,      a_s = a(t + c_s h, x_s),
and the step ends with
    x_new = x + h v + h^2 sum_m (b A)_m a_m,             v_new = v + h sum_m b_m a_m,
    e_x   = h^2 sum_m ((b - bhat) A)_m a_m,              e_v   = h sum_m (b - bhat)_m a_m,
(sum_m (b - bhat)_m = 0 removes the v term of e_x). The continuous extension
y(t + s h) = y + h sum_j b_j(s) k_j becomes
    x(s) = x + s h v + h^2 sum_m P_m(s) a_m,  P_m(s) = sum_j b_j(s) A_jm,    v(s) = v + h sum_j b_j(s) a_j.
This is exact algebra on the published tableau (Dormand & Prince 1980; continuous extension of
Shampine 1986 as used by ode45); only the rounding order differs from the textbook form.
Every coefficient is computed here in exact rational arithmetic and printed correctly rounded.
"""
from fractions import Fraction as F
import os

C = [F(0), F(1, 5), F(3, 10), F(4, 5), F(8, 9), F(1), F(1)]
A = [[F(0)] * 7 for _ in range(7)]
A[1][0] = F(1, 5)
A[2][0], A[2][1] = F(3, 40), F(9, 40)
A[3][0], A[3][1], A[3][2] = F(44, 45), F(-56, 15), F(32, 9)
A[4][0], A[4][1], A[4][2], A[4][3] = F(19372, 6561), F(-25360, 2187), F(64448, 6561), F(-212, 729)
A[5][0], A[5][1], A[5][2], A[5][3], A[5][4] = (F(9017, 3168), F(-355, 33), F(46732, 5247),
                                               F(49, 176), F(-5103, 18656))
A[6][0], A[6][1], A[6][2], A[6][3], A[6][4], A[6][5] = (F(35, 384), F(0), F(500, 1113),
                                                         F(125, 192), F(-2187, 6784), F(11, 84))
B = A[6][:]
BHAT = [F(5179, 57600), F(0), F(7571, 16695), F(393, 640), F(-92097, 339200), F(187, 2100), F(1, 40)]
BI = [[F(1), F(-183, 64), F(37, 12), F(-145, 128)],
      [F(0)] * 4,
      [F(0), F(1500, 371), F(-1000, 159), F(1000, 371)],
      [F(0), F(-125, 32), F(125, 12), F(-375, 64)],
      [F(0), F(9477, 3392), F(-729, 106), F(25515, 6784)],
      [F(0), F(-11, 7), F(11, 3), F(-55, 28)],
      [F(0), F(3, 2), F(-4), F(5, 2)]]

for i in range(7):
    assert sum(A[i]) == C[i]
assert sum(B) == 1 and sum(BHAT) == 1
E = [B[i] - BHAT[i] for i in range(7)]
AA = [[sum(A[s][l] * A[l][m] for l in range(7)) for m in range(7)] for s in range(7)]
EA = [sum(E[l] * A[l][m] for l in range(7)) for m in range(7)]
P = [[sum(BI[j][p] * A[j][m] for j in range(7)) for p in range(4)] for m in range(7)]
for j in range(7):
    assert sum(BI[j]) == B[j]


def lit(x):
    return repr(float(x))


lines = ["// Generated by gen_dp5_nystrom.py from the Dormand-Prince 5(4) tableau. Do not edit.",
         "#pragma once", ""]
lines.append("// stage nodes c_s")
for s in range(7):
    lines.append(f"#define DP_C{s + 1} {lit(C[s])}")
lines.append("// (A A)_{sm}: h^2 weights of accelerations in stage positions (stage s = 1..7, m = 1..s-2)")
for s in range(7):
    for m in range(7):
        if AA[s][m] != 0:
            lines.append(f"#define DP_AA{s + 1}{m + 1} {lit(AA[s][m])}")
lines.append("// b: fifth-order velocity weights (b2 = b7 = 0)")
for m in range(7):
    if B[m] != 0:
        lines.append(f"#define DP_B{m + 1} {lit(B[m])}")
lines.append("// b - bhat: embedded error weights on accelerations (velocity error)")
for m in range(7):
    if E[m] != 0:
        lines.append(f"#define DP_E{m + 1} {lit(E[m])}")
lines.append("// (b - bhat) A: embedded error weights on accelerations (position error, times h^2)")
for m in range(7):
    if EA[m] != 0:
        lines.append(f"#define DP_EA{m + 1} {lit(EA[m])}")
lines.append("// continuous extension: velocity weights b_j(s) = sum_p BI_jp s^(p+1)")
for j in range(7):
    for p in range(4):
        if BI[j][p] != 0:
            lines.append(f"#define DP_BI{j + 1}{p + 1} {lit(BI[j][p])}")
lines.append("// continuous extension: position weights P_m(s) = sum_p PX_mp s^(p+1), times h^2")
for m in range(7):
    for p in range(4):
        if P[m][p] != 0:
            lines.append(f"#define DP_PX{m + 1}{p + 1} {lit(P[m][p])}")
out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dp5_nystrom.h")
with open(out, "w") as f:
    f.write("\n".join(lines) + "\n")
print("wrote", out)
