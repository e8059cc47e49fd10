"""50-digit brute force of the per-pair path bin and weight (Eq. 1 generalised
to laser/detector spots, stand-off legs and Lambertian cosines), used only to
pin the FP64 oracle on tiny grids. Pure Python ``decimal``; slow by design.
"""
from decimal import Decimal, getcontext

import numpy as np

getcontext().prec = 50
C = Decimal(299792458)


def _D(x) -> Decimal:
    return Decimal(float(x))  # exact binary value of the (float32 -> float64) input


def _norm(v):
    return (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]).sqrt()


def bruteforce_pairs(params, pts):
    nx, ny = int(params["scan_nx"]), int(params["scan_ny"])
    wx, wy = _D(params["wall_half_x"]), _D(params["wall_half_y"])
    h = _D(params["standoff_m"])
    dt = _D(params["bin_width_s"])
    ws = float(params["window_start_m"])
    L0 = 2 * h if ws != ws else _D(ws)
    mode = params["cos_mode"]
    S = nx * ny
    P = pts.shape[0]
    u_out = np.zeros((S, P))
    w_out = np.zeros((S, P))
    for s in range(S):
        ix, iy = s % nx, s // nx
        dx = -wx + (Decimal(ix) + Decimal("0.5")) * (2 * wx / nx)
        dy = -wy + (Decimal(iy) + Decimal("0.5")) * (2 * wy / ny)
        d = (dx, dy, Decimal(0))
        if params["scan_mode"] == "nonconfocal":
            lv = (_D(params["laser_xy"][0]), _D(params["laser_xy"][1]), Decimal(0))
        else:
            lv = d
        if params["standoff_mode"] == "constant":
            legs = 2 * h
        else:
            legs = (lv[0] ** 2 + lv[1] ** 2 + h * h).sqrt() + (d[0] ** 2 + d[1] ** 2 + h * h).sqrt()
        for q in range(P):
            x = [_D(v) for v in pts[q, 0:3]]
            n = [_D(v) for v in pts[q, 3:6]]
            rho, area = _D(pts[q, 6]), _D(pts[q, 7])
            vl = [x[i] - lv[i] for i in range(3)]
            vd = [x[i] - d[i] for i in range(3)]
            rl, rd = _norm(vl), _norm(vd)
            u = (legs + rl + rd - L0) / (C * dt)
            cf = Decimal(1)
            if mode in ("object", "object_wall"):
                cl = -(n[0] * vl[0] + n[1] * vl[1] + n[2] * vl[2]) / rl
                cd = -(n[0] * vd[0] + n[1] * vd[1] + n[2] * vd[2]) / rd
                cf = max(cl, Decimal(0)) * max(cd, Decimal(0))
                if mode == "object_wall":
                    cf *= (vl[2] / rl) * (vd[2] / rd)
            w = rho * area * cf / (rl * rl * rd * rd)
            u_out[s, q] = float(u)
            w_out[s, q] = float(w)
    return u_out, w_out
