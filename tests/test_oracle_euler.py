"""Pins of the Euler finite-volume oracle (oracle/euler.py) against what the
mathematics fixes, none of which compares the oracle with itself:

  * exact Riemann solver: the Rankine-Hugoniot conditions across its shocks,
    the Riemann invariants across its rarefactions and the equality of
    pressure and velocity across its contact; the star state of Sod's problem
    (p* = 0.30313, u* = 0.92745, the textbook figures);
  * uniform states are preserved bit for bit (every face flux is the same);
  * mass, momentum and energy are conserved to rounding on the periodic grid;
  * a y-uniform Sod problem stays y-uniform bit for bit and converges to the
    exact Riemann solution (L1 error of density falling with the cell
    count; no new extrema);
  * the isentropic vortex converges at second order (observed order >= 1.4
    between 32, 64 and 128 cells; a first-order scheme gives 1), and at
    second order in time on a fixed grid (error ratio >= 3 when dt halves;
    a first-order integrator gives 2);
  * a quarter turn and a mirror image commute with the step;
  * the time step is the CFL formula evaluated cell by cell.
Planted mistakes (in the oracle, on the CPU) each fail one of these.
"""
import numpy as np
import pytest

from oracle import euler as E

SOD_L = (1.0, 0.0, 1.0)
SOD_R = (0.125, 0.0, 0.1)


def sod_state(N, ny=4):
    """Periodic double Sod problem: the left state on [1/4, 3/4), the right
    state elsewhere; two mirror-image Riemann problems that do not meet
    before t = 0.14."""
    x = (np.arange(N) + 0.5) / N
    inside = (x >= 0.25) & (x < 0.75)
    rho = np.where(inside, SOD_L[0], SOD_R[0])
    p = np.where(inside, SOD_L[2], SOD_R[2])
    W = np.stack([np.tile(rho, (ny, 1)), np.zeros((ny, N)), np.zeros((ny, N)), np.tile(p, (ny, 1))])
    return E.conserved(W), x


def run_to(U, dx, dy, tf, cfl=0.4, mod=E):
    t = 0.0
    while t < tf - 1e-15:
        dt = min(cfl / mod.max_wave(U, dx, dy), tf - t)
        U, _ = mod.step(U, dx, dy, dt=dt)
        t += dt
    return U


def sod_error(N, mod=E, tf=0.1):
    U, x = sod_state(N)
    U = run_to(U, 1.0 / N, 1.0 / N, tf, mod=mod)
    right = E.exact_riemann(SOD_L, SOD_R, (x - 0.75) / tf)[0]
    left = E.exact_riemann(SOD_L, SOD_R, (0.25 - x) / tf)[0]
    exact = np.where(x >= 0.5, right, left)
    return float(np.mean(np.abs(U[0, 0] - exact))), U


def vortex_error(N, mod=E, tf=1.0):
    L = 10.0
    U = run_to(E.isentropic_vortex(N, N), L / N, L / N, tf, mod=mod)
    return float(np.mean(np.abs(U[0] - E.isentropic_vortex(N, N, t=tf)[0])))


def random_state(rng, ny, nx, amp=0.3):
    """A smooth-ish positive state: rho, p in [1 - amp, 1 + amp], |u|, |v| <= amp."""
    rho = 1.0 + amp * rng.uniform(-1, 1, (ny, nx))
    p = 1.0 + amp * rng.uniform(-1, 1, (ny, nx))
    u = amp * rng.uniform(-1, 1, (ny, nx))
    v = amp * rng.uniform(-1, 1, (ny, nx))
    return E.conserved(np.stack([rho, u, v, p]))


# ------------------------------------------------------------------ exact Riemann solver
def test_sod_star_state():
    p, u = E.star_state(SOD_L, SOD_R)
    assert abs(p - 0.30313) < 1e-5 and abs(u - 0.92745) < 1e-5


@pytest.mark.parametrize("WL,WR", [(SOD_L, SOD_R), ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01)),
                                   ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4)),
                                   ((5.99924, 19.5975, 460.894), (5.99242, -6.19633, 46.095))])
def test_exact_riemann_jump_conditions(WL, WR):
    g = E.GAMMA
    ps, us = E.star_state(WL, WR, g)
    xi = np.linspace(-40, 40, 40001)
    r, u, p = E.exact_riemann(WL, WR, xi, g)
    # far field
    assert (r[0], u[0], p[0]) == WL and (r[-1], u[-1], p[-1]) == WR
    # across the contact pressure and velocity are continuous
    k = np.searchsorted(xi, us)
    assert abs(p[k - 2] - ps) < 1e-9 * ps and abs(p[k + 2] - ps) < 1e-9 * ps
    assert abs(u[k - 2] - us) < 1e-9 * (1 + abs(us)) and abs(u[k + 2] - us) < 1e-9 * (1 + abs(us))
    for side, (rk, uk, pk) in ((-1, WL), (1, WR)):
        rs = r[k - 2] if side < 0 else r[k + 2]
        if ps > pk:
            # shock: mass, momentum and energy fluxes equal in the shock frame
            S = (rs * us - rk * uk) / (rs - rk)
            m1, m2 = rk * (uk - S), rs * (us - S)
            assert abs(m1 - m2) < 1e-9 * (abs(m1) + 1e-300)
            assert abs((m1 * (uk - S) + pk) - (m2 * (us - S) + ps)) < 1e-9 * (abs(pk) + abs(ps))
            h1 = g / (g - 1) * pk / rk + 0.5 * (uk - S) ** 2
            h2 = g / (g - 1) * ps / rs + 0.5 * (us - S) ** 2
            assert abs(h1 - h2) < 1e-9 * h1
        else:
            # rarefaction: entropy and the Riemann invariant u -+ 2c/(g-1) constant
            assert abs(ps / rs**g - pk / rk**g) < 1e-9 * pk / rk**g
            ck, cs = np.sqrt(g * pk / rk), np.sqrt(g * ps / rs)
            J = uk - side * 2 * ck / (g - 1)
            assert abs((us - side * 2 * cs / (g - 1)) - J) < 1e-9 * (1 + abs(J))
            # inside the fan too
            lo, hi = (uk - ck, us - cs) if side < 0 else (us + cs, uk + ck)
            fan = (xi > lo + 1e-3) & (xi < hi - 1e-3)
            if fan.any():
                cf = np.sqrt(g * p[fan] / r[fan])
                assert np.allclose(p[fan] / r[fan] ** g, pk / rk**g, rtol=1e-9)
                assert np.allclose(u[fan] - side * 2 * cf / (g - 1), J, rtol=0, atol=1e-9 * (1 + abs(J)))


# ------------------------------------------------------------------ the scheme
def test_uniform_state_is_preserved_bitwise():
    W = np.stack([np.full((6, 10), 1.3), np.full((6, 10), 0.7), np.full((6, 10), -0.2),
                  np.full((6, 10), 2.1)])
    U = E.conserved(W)
    U2, dt = E.step(U, 0.1, 0.2)
    assert dt > 0 and np.array_equal(U2, U)


def test_conservation_to_rounding():
    rng = np.random.default_rng(1)
    U = random_state(rng, 24, 40)
    s0 = U.sum(axis=(1, 2))
    U2, _ = E.run(U, 0.05, 0.04, 10)
    s1 = U2.sum(axis=(1, 2))
    assert np.all(np.abs(s1 - s0) <= 1e-12 * np.abs(U).sum(axis=(1, 2)))


def test_sod_reduction_to_the_exact_riemann_solution():
    e200, _ = sod_error(200)
    e400, U = sod_error(400)
    assert e400 < 0.008 and e400 < 0.75 * e200
    # y-uniform data stays y-uniform bit for bit; no new extrema of density
    assert all(np.array_equal(U[:, 0], U[:, j]) for j in range(1, U.shape[1]))
    assert U[0].min() >= SOD_R[0] - 1e-12 and U[0].max() <= SOD_L[0] + 1e-12


def test_vortex_second_order():
    e = [vortex_error(n) for n in (32, 64, 128)]
    o1, o2 = np.log2(e[0] / e[1]), np.log2(e[1] / e[2])
    assert o1 >= 1.4 and o2 >= 1.4, (e, o1, o2)


def time_order_ratio(mod=E):
    """Error ratio of dt = 0.01 over dt = 0.005 against dt = 0.00125 on the
    32^2 vortex at t = 0.5 (fixed steps below the CFL limit)."""
    N, L = 32, 10.0
    h = L / N
    U0 = E.isentropic_vortex(N, N)

    def fixed(dt):
        U = U0
        for _ in range(int(round(0.5 / dt))):
            U, _ = mod.step(U, h, h, dt=dt)
        return U
    ref = fixed(0.00125)
    return np.max(np.abs(fixed(0.01) - ref)) / np.max(np.abs(fixed(0.005) - ref))


def test_time_integration_second_order():
    assert time_order_ratio() >= 3.0


def test_quarter_turn_and_mirror_commute_with_the_step():
    rng = np.random.default_rng(2)
    U = random_state(rng, 20, 20)
    h = 0.05
    U2, dt = E.step(U, h, h)

    def turn(V):  # (x, y) -> (y, x): swap the axes and the velocities
        return np.stack([V[0].T, V[2].T, V[1].T, V[3].T])

    T2, dtt = E.step(turn(U), h, h)
    assert dtt == dt
    assert np.max(np.abs(T2 - turn(U2))) <= 1e-13 * np.max(np.abs(U2))

    def mirror(V):  # x -> -x: reverse x, negate u
        return np.stack([V[0][:, ::-1], -V[1][:, ::-1], V[2][:, ::-1], V[3][:, ::-1]])

    M2, _ = E.step(mirror(U), h, h)
    assert np.max(np.abs(M2 - mirror(U2))) <= 1e-13 * np.max(np.abs(U2))


def test_time_step_cell_by_cell():
    rng = np.random.default_rng(3)
    U = random_state(rng, 5, 7)
    dx, dy, g = 0.3, 0.2, E.GAMMA
    best = 0.0
    for j in range(5):
        for i in range(7):
            rho, mx, my, en = U[:, j, i]
            u, v = mx / rho, my / rho
            p = (g - 1) * (en - 0.5 * rho * (u * u + v * v))
            c = (g * p / rho) ** 0.5
            best = max(best, (abs(u) + c) / dx + (abs(v) + c) / dy)
    assert abs(E.max_wave(U, dx, dy) - best) <= 1e-15 * best
    _, dt = E.step(U, dx, dy, cfl=0.4)
    assert dt == 0.4 / E.max_wave(U, dx, dy)


# ------------------------------------------------------------------ planted mistakes
class Mutant:
    """A copy of the oracle's module namespace with one function replaced."""

    def __init__(self, **repl):
        import types
        self.mod = types.ModuleType("euler_mutant")
        self.mod.__dict__.update({k: v for k, v in E.__dict__.items() if not k.startswith("__")})
        self.mod.__dict__.update(repl)
        # rebind the module-level functions' globals to the mutant namespace
        for k, v in list(self.mod.__dict__.items()):
            if callable(v) and getattr(v, "__module__", None) == E.__name__ and k not in repl:
                self.mod.__dict__[k] = types.FunctionType(v.__code__, self.mod.__dict__, k,
                                                          v.__defaults__)
        for k in repl:
            f = repl[k]
            self.mod.__dict__[k] = types.FunctionType(f.__code__, self.mod.__dict__, k, f.__defaults__)


def _central_slopes(W, axis):
    return 0.5 * (np.roll(W, -1, axis=axis) - np.roll(W, 1, axis=axis))


def _wrong_normal_flux(W, axis, gamma=1.4):
    rho, u, v, p = W
    un = u                                     # uses u on y faces too
    E_ = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho * un, rho * un * u + (p if axis == 2 else 0.0),
                     rho * un * v + (p if axis == 1 else 0.0), un * (E_ + p)])


def _wrong_gamma_primitives(U, gamma=1.4):
    rho = U[0]
    u, v = U[1] / rho, U[2] / rho
    return np.stack([rho, u, v, (5.0 / 3.0 - 1.0) * (U[3] - 0.5 * rho * (u * u + v * v))])


def _forward_euler_step(U, dx, dy, cfl=0.4, dt=None, gamma=1.4):
    if dt is None:
        dt = cfl / max_wave(U, dx, dy, gamma)  # noqa: F821 (mutant namespace)
    return U + dt * rhs(U, dx, dy, gamma), dt  # noqa: F821


def _no_upwind_term(WL, WR, axis, gamma=1.4):
    return 0.5 * (physical_flux(WL, axis, gamma) + physical_flux(WR, axis, gamma))  # noqa: F821


def _first_order_states(W, s, axis):
    return W, np.roll(W, -1, axis=axis)


def _fails_a_pin(mod):
    try:
        e, U = sod_error(200, mod=mod)
        if not (e < 0.012) or U[0].max() > SOD_L[0] + 1e-12 or U[0].min() < SOD_R[0] - 1e-12:
            return True
        e32, e64 = vortex_error(32, mod=mod), vortex_error(64, mod=mod)
        if not np.log2(e32 / e64) >= 1.4:
            return True
        if not time_order_ratio(mod) >= 3.0:
            return True
        rng = np.random.default_rng(2)
        U = random_state(rng, 12, 12)
        U2, _ = mod.step(U, 0.05, 0.05)
        tr = lambda V: np.stack([V[0].T, V[2].T, V[1].T, V[3].T])  # noqa: E731
        T2, _ = mod.step(tr(U), 0.05, 0.05)
        return np.max(np.abs(T2 - tr(U2))) > 1e-13 * np.max(np.abs(U2))
    except (FloatingPointError, ValueError, OverflowError):
        return True


@pytest.mark.parametrize("name,repl", [
    ("central slopes (no limiter)", {"slopes": _central_slopes}),
    ("u as the normal velocity of y faces", {"physical_flux": _wrong_normal_flux}),
    ("gamma 5/3 in the primitives", {"primitives": _wrong_gamma_primitives}),
    ("forward Euler instead of RK2", {"step": _forward_euler_step}),
    ("no upwind term in the flux", {"rusanov": _no_upwind_term}),
    ("first-order face states", {"face_states": _first_order_states}),
])
def test_planted_mistakes_fail_a_pin(name, repl):
    with np.errstate(all="ignore"):
        assert _fails_a_pin(Mutant(**repl).mod), name


def test_the_unmodified_oracle_passes_the_mutant_screen():
    with np.errstate(all="ignore"):
        assert not _fails_a_pin(Mutant().mod)
