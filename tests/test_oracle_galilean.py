"""The coupled free-sphere loop at steady state, pinned by Galilean
invariance (Sect. 2.3 with the DEM of Sect. 2.1).

A free sphere of radius 2.5 between two walls at rest (x, y periodic),
pushed along x by a constant external force F, reaches a terminal velocity
V_t: the moving-boundary bounce-back (Eqs. 19-21), the momentum exchange
(Eq. 25), the refill of uncovered nodes and the Verlet update all act on
it.  In the frame that moves with it the same flow is a fixed sphere with
both walls, and the fluid far from it, moving at -V_t; the steady drag on
that fixed sphere must then balance F.  BGK is Galilean invariant up to the
O(u^3) terms the second-order equilibrium drops, and the moving sphere
samples every sub-node position while the fixed one sits at one, so the two
agree to a fraction of a percent (0.4% observed, V_t = 0.0056, Mach 0.01);
the test allows 1%.  A weight error in the moving-boundary term moves V_t
well off this balance: planted in a copy of the oracle, half the term in
the q < 1/2 branch, or twice it in the q >= 1/2 branch, leaves the drag
about 40% away from F (the second test plants the first).  Both runs start
from their own steady far field (rest; uniform -V_t) and take 1500 steps,
past the channel's viscous time h^2 / nu = 1536.
"""
import numpy as np

import oracle

BOX = (24, 24, 16)
TAU, R, F0 = 1.0, 2.5, 0.05
X0 = np.array([[12.3, 12.1, 7.5]])  # mid-height: no lift, no torque by symmetry
STEPS, AVG = 1500, 500


def terminal_velocity():
    """Velocities of the free sphere over the last AVG steps."""
    nx, ny, nz = BOX
    free = oracle.Oracle(nx, ny, nz, TAU, cs=0.0, rho_s=2.5)
    free.set_particles(X0, R=[R])
    free.set_load(F=np.array([[F0, 0.0, 0.0]]))
    V = []
    for k in range(STEPS):
        free.step(1)
        if k >= STEPS - AVG:
            V.append(free.particles()[1][0].copy())
    z = free.particles()[0][0, 2]
    free.close()
    return np.array(V), z


def co_moving_drag(vt):
    """Mean force over the last AVG steps on the sphere held fixed, walls and
    far field moving at -vt."""
    nx, ny, nz = BOX
    fixed = oracle.Oracle(nx, ny, nz, TAU, cs=0.0, rho_s=2.5, u_lo=(-vt, 0.0, 0.0), u_hi=(-vt, 0.0, 0.0))
    fq = oracle.feq(1.0, [-vt, 0.0, 0.0])
    fixed.set_populations(np.broadcast_to(fq[:, None, None, None], (19, nz, ny, nx)))
    fixed.set_particles(X0, R=[R], fixed=[1])
    D = []
    for k in range(STEPS):
        fixed.step(1)
        if k >= STEPS - AVG:
            D.append(fixed.forces()[0][0].copy())
    fixed.close()
    return np.array(D).mean(axis=0)


def test_free_sphere_terminal_velocity_balances_the_co_moving_fixed_drag():
    V, z = terminal_velocity()
    vt = V[:, 0].mean()
    assert vt > 0.0
    assert np.abs(V[:, 1:].mean(axis=0)).max() < 1e-3 * vt  # along x on average (y sees the lattice)
    assert abs(z - X0[0, 2]) < 1e-9  # stays at mid-height
    D = co_moving_drag(vt)
    # the fluid drags the fixed sphere along -x with the force that held the free one
    assert abs(-D[0] - F0) <= 1e-2 * F0
    assert np.abs(D[1:]).max() < 1e-3 * F0


def test_a_planted_weight_error_in_the_moving_boundary_term_breaks_the_balance(tmp_path):
    src = oracle.source()
    term = "double dw = 6.0 * s->w[j] * cku;"
    assert src.count(term) == 1
    with oracle.Planted(src.replace(term, "double dw = 3.0 * s->w[j] * cku;"), tmp_path / "planted.so"):
        V, _ = terminal_velocity()
        D = co_moving_drag(V[:, 0].mean())
    assert abs(-D[0] - F0) > 0.2 * F0
