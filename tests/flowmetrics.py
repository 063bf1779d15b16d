"""Measurements the tests take on a solution (from any implementation): primitive variables, the closed-form
oblique-shock relations and the shock angle / pressure ratio measured over the wedge (Sec. 8.1.6 workload)."""
import math

import numpy as np

GAMMA = 1.4


def prim(U, gamma=GAMMA):
    r, mx, my, E = U
    u, v = mx / r, my / r
    return r, u, v, (gamma - 1.0) * (E - 0.5 * r * (u * u + v * v))


def theta_beta_m(M, theta, g=GAMMA):
    """Weak-branch shock angle of the theta-beta-M relation and the normal-shock pressure ratio behind it."""
    from scipy.optimize import brentq

    def f(b):
        return math.tan(theta) - 2.0 / math.tan(b) * (M * M * math.sin(b) ** 2 - 1) / (
            M * M * (g + math.cos(2 * b)) + 2)

    mu = math.asin(1.0 / M)
    beta = brentq(f, mu + 1e-9, mu + 0.5 * (math.pi / 2 - mu))
    Mn = M * math.sin(beta)
    return beta, 1.0 + 2.0 * g / (g + 1) * (Mn * Mn - 1)


def theta_from_beta(M, beta, g=GAMMA):
    """Wedge angle (deg) whose attached oblique shock stands at beta (radians): the theta-beta-M relation solved
    for theta."""
    t = 2.0 / math.tan(beta) * (M * M * math.sin(beta) ** 2 - 1) / (M * M * (g + math.cos(2 * beta)) + 2)
    return math.degrees(math.atan(t))


def theta_from_ratio(M, ratio, g=GAMMA):
    """Wedge angle (deg) whose weak oblique shock has the pressure ratio p2/p1 = ratio."""
    Mn2 = 1.0 + (ratio - 1.0) * (g + 1) / (2.0 * g)
    return theta_from_beta(M, math.asin(math.sqrt(Mn2) / M), g)


def wedge_shock(U, tags, spec, xs=(0.45, 0.55, 0.65, 0.75)):
    """Angle (deg) and pressure ratio of the shock above the wedge's upper face: on each column x in xs the
    height where p crosses the mean of the free-stream and theta-beta-M post-shock pressures (linear between
    cells), the angle from the slope of a line through those points (the slope, not the position: the
    immersed no-slip wall shifts the effective leading edge by a few cells), the ratio from the median
    pressure between the wall (3 cells off) and the shock (2 cells off) over the free-stream pressure."""
    nx, ny = spec["nx"], spec["ny"]
    x0, x1, y0, y1 = spec["domain"]
    _, _, _, p = prim(U, spec["gamma"])
    xc = x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx
    yc = y0 + (np.arange(ny) + 0.5) * (y1 - y0) / ny
    _, pr_e = theta_beta_m(spec["mach"], math.radians(15.0), spec["gamma"])
    p1 = 1.0 / (spec["gamma"] * spec["mach"] ** 2)
    mid = p1 * (1.0 + pr_e) / 2.0
    px, py, plateau = [], [], []
    for xt in xs:
        i = int(np.argmin(np.abs(xc - xt)))
        col = p[:, i]
        j = max(jj for jj in range(ny - 1) if col[jj] >= mid and col[jj + 1] < mid)
        py.append(yc[j] + (col[j] - mid) / (col[j] - col[j + 1]) * (yc[j + 1] - yc[j]))
        px.append(xc[i])
        wall = max(jj for jj in range(ny) if tags[jj, i] != 0)
        plateau.append(np.median(col[wall + 3:j - 2]) / p1)
    slope = np.polyfit(px, py, 1)[0]
    return math.degrees(math.atan(slope)), float(np.median(plateau))


def deviation_error(a, b, live, uinf_state):
    """Largest difference per conserved variable over live cells, relative to the largest deviation of b from
    the free stream (the scale of what the flow computed)."""
    out = []
    for k in range(4):
        dev = np.abs(b[k] - uinf_state[k])[live].max()
        out.append(float(np.abs(a[k] - b[k])[live].max() / max(dev, 1e-300)))
    return out


def rel_state_error(a, b, tags):
    """Largest |a - b| / max(1, |b|) over the conserved variables of non-solid cells."""
    live = tags != 1
    return float(np.max(np.abs(a - b)[:, live] / np.maximum(1.0, np.abs(b)[:, live])))


def ulp_floor(orc, spec, nsteps, state=None):
    """The oracle's own sensitivity: how far its state moves (in the measure of rel_state_error) after nsteps when the
    initial total energy of every cell moves by one unit in the last place.  At low Mach the absolute FP64
    energy rho E ~ p_inf / (gamma - 1) = 1 / (gamma (gamma - 1) M^2) holds the pressure fluctuation p' only to
    eps p_inf, and the preconditioned scheme turns pressure differences into velocity differences through the
    impedance rho U_r with U_r of the order of the flow speed, not the sound speed: two correct FP64 codes that
    round differently (contraction, reciprocals) drift apart at this rate (measured 2e-9 at M = 0.001 and 5e-11
    at M = 0.01 on a cylinder at 8 cells per diameter after 6 steps of 10 sub-iterations)."""
    a, b = orc.Case(spec), orc.Case(spec)
    U = a.state() if state is None else np.array(state, dtype=np.float64)
    if state is not None:
        a.set_state(U)
    rng = np.random.default_rng(5)
    Up = U.copy()
    Up[3] = np.nextafter(U[3], np.where(rng.random(U[3].shape) < 0.5, np.inf, -np.inf))
    b.set_state(Up)
    a.step(nsteps)
    b.step(nsteps)
    return rel_state_error(b.state(), a.state(), a.tags())


def fp64_bar(orc, spec, nsteps, state=None):
    """Bar of an FP64 state comparison with the oracle: 1e-10 relative, or four times the oracle's own
    one-ulp sensitivity where that is larger."""
    return max(1e-10, 4.0 * ulp_floor(orc, spec, nsteps, state))
