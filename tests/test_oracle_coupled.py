"""Pins of the oracle's body motion under the fluid force (Sec. 6, Eq. 10; the shock-driven cylinder of
Sec. 8.2.6).

The integrator is pinned by what the mechanics fixes rather than by its own
formula: an infinitely heavy body reproduces the fixed body; a body carried by
a uniform stream feels no force and keeps its velocity; over every step the
displacement is the trapezoidal integral of the velocity (exact for the
step's constant acceleration, which the printed update without the factor 1/2
would break); the momentum gained equals the impulse of the recorded forces;
and the mirror-symmetric shock-driven cylinder feels no transverse force.
"""
import numpy as np

from paper_1912_11908_gb300 import workloads as W


def _shock_case(orc, res=16, **kw):
    spec = W.shock_driven_cylinder(4 * res, 4 * res, **kw)
    c = orc.Case(spec)
    c.set_state(W.shock_initial_state(spec))
    return spec, c


def test_infinitely_heavy_body_is_the_fixed_body(orc):
    """mass -> infinity: the shock passes a body that does not move; state and forces equal the static body's."""
    spec, heavy = _shock_case(orc, density_ratio=1e300)
    fixed = orc.Case(dict(spec, motion=W.MOTION_STATIC))
    fixed.set_state(W.shock_initial_state(spec))
    for _ in range(4):
        heavy.step(20)
        fixed.step(20)
    assert heavy.time() > 0.6  # the shock has hit the body
    b = heavy.body()
    assert np.all(np.abs(b[:4]) < 1e-290)
    np.testing.assert_array_equal(heavy.tags(), fixed.tags())
    a, f = heavy.state(), fixed.state()
    assert np.abs(a - f).max() <= 1e-13 * np.abs(f).max()
    np.testing.assert_allclose(heavy.forces(), fixed.forces(), rtol=0, atol=1e-13)


def test_body_carried_by_a_uniform_stream_keeps_its_velocity(orc):
    """A free body moving with the uniform stream feels no force: velocity and the uniform field are kept while
    it is re-classified every step, and its displacement is velocity x time."""
    spec = W.case_spec(W.cylinder(64, 1.0), 96, 48, (-2.0, 6.0, -2.0, 2.0), 0.5, 100.0, W.FAR,
                       motion=W.MOTION_COUPLED, vel=(1.0, 0.0), mass=0.5)
    c = orc.Case(spec)
    U0 = c.state()
    c.step(60)
    t = c.time()
    assert t > 0.4  # several cells crossed
    b = c.body()
    assert abs(b[2] - 1.0) < 1e-12 and abs(b[3]) < 1e-12
    assert abs(b[0] - t) < 1e-12 and abs(b[1]) < 1e-12
    U1 = c.state()
    live = c.tags() != 1
    for k in range(4):
        assert np.abs(U1[k] - U0[k])[live].max() <= 1e-12 * max(1.0, np.abs(U0[k]).max()), k


def test_trajectory_is_the_integral_of_velocity_and_impulse(orc):
    """Step by step through the shock's impact: x_{n+1} - x_n = (u_n + u_{n+1}) dt_n / 2 and
    M (u_N - u_0) = sum F_n dt_n; the body is pushed downstream and feels no transverse force."""
    spec, c = _shock_case(orc, density_ratio=2.0)
    M = spec["mass"]
    b0 = c.body()
    prev = b0
    impulse = np.zeros(2)
    fmax = 0.0
    for _ in range(150):
        c.step(1)
        dt = c.last_dt()
        b = c.body()
        for d in range(2):
            disp = b[d] - prev[d]
            assert abs(disp - 0.5 * (prev[2 + d] + b[2 + d]) * dt) <= 1e-15 + 1e-13 * abs(disp)
        impulse += b[4:6] * dt
        fmax = max(fmax, abs(b[4]))
        assert abs(b[5]) <= 1e-9 * max(fmax, 1e-3)  # mirror symmetry about the centre line
        prev = b
    assert c.time() > 1.0
    np.testing.assert_allclose(M * (prev[2:4] - b0[2:4]), impulse, rtol=1e-12, atol=1e-15)
    assert prev[2] > 0.05 and prev[0] > 0.01  # pushed along the shock's direction
