"""FP64 oracle of the 2D Euler finite-volume step.

TEST INFRASTRUCTURE ONLY (tests/, the smoke check, the benchmark's CPU legs).

The paper's second workload (Sec. IV, the Euler result of Fig. "Euler"; Sec.
V) is a finite-volume solver of the 2D Euler equations of gas dynamics built
from "many different types of stencil and pointwise operations", fused by
ProtoX against Proto's operator-by-operator code. The paper names no scheme;
this oracle takes the textbook second-order one, written as the separate
passes an operator library composes:

  state     U = (rho, rho u, rho v, E) cell averages on a periodic nx x ny grid
            (arrays shaped (4, ny, nx), x fastest), ideal gas
            p = (gamma - 1) (E - rho (u^2 + v^2) / 2);
  pass 1    primitives W = (rho, u, v, p) of every cell;
  pass 2    limited slopes per direction, s_i = minmod(W_i - W_{i-1}, W_{i+1} - W_i),
            minmod(a, b) = 0 if a b <= 0, else the one of smaller magnitude;
  pass 3    face states W_L = W_i + s_i / 2, W_R = W_{i+1} - s_{i+1} / 2 at the
            face i + 1/2 (likewise in y);
  pass 4    Rusanov (local Lax-Friedrichs) flux
            F = (F(W_L) + F(W_R)) / 2 - a (U(W_R) - U(W_L)) / 2,
            a = max(|u_n,L| + c_L, |u_n,R| + c_R), c = sqrt(gamma p / rho),
            F(W) = (rho u_n, rho u_n u + p n_x, rho u_n v + p n_y, u_n (E + p));
  pass 5    divergence L(U)_ij = -(F_{i+1/2} - F_{i-1/2}) / dx - (G_{j+1/2} - G_{j-1/2}) / dy;
  pass 6    SSP Runge-Kutta 2 (Heun): U1 = U + dt L(U), U' = (U + U1 + dt L(U1)) / 2;
  pass 7    time step from the max wave speed of the state the step starts from,
            dt = cfl / max_cells((|u| + c) / dx + (|v| + c) / dy).

The exact Riemann solver (exact_riemann) is the standard two-rarefaction /
shock construction for the ideal-gas Riemann problem (Newton iteration for
the star pressure, then sampling of the self-similar solution); it serves the
pins, not the scheme.
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


# ------------------------------------------------------------------ pass 1
def primitives(U, gamma=GAMMA):
    rho = U[0]
    u = U[1] / rho
    v = U[2] / rho
    p = (gamma - 1.0) * (U[3] - 0.5 * rho * (u * u + v * v))
    return np.stack([rho, u, v, p])


def conserved(W, gamma=GAMMA):
    rho, u, v, p = W
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


# ------------------------------------------------------------------ pass 2
def minmod(a, b):
    return np.where(a * b <= 0.0, 0.0, np.where(np.abs(a) < np.abs(b), a, b))


def slopes(W, axis):
    """Limited slope of every cell along axis (2 = x, 1 = y), periodic."""
    back = W - np.roll(W, 1, axis=axis)      # W_i - W_{i-1}
    fwd = np.roll(W, -1, axis=axis) - W      # W_{i+1} - W_i
    return minmod(back, fwd)


# ------------------------------------------------------------------ pass 3
def face_states(W, s, axis):
    """(W_L, W_R) at the face i + 1/2 of every cell i along axis."""
    WL = W + 0.5 * s
    WR = np.roll(W - 0.5 * s, -1, axis=axis)
    return WL, WR


# ------------------------------------------------------------------ pass 4
def physical_flux(W, axis, gamma=GAMMA):
    """Flux of U through a face whose normal is x (axis 2) or y (axis 1)."""
    rho, u, v, p = W
    un = u if axis == 2 else v
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho * un,
                     rho * un * u + (p if axis == 2 else 0.0),
                     rho * un * v + (p if axis == 1 else 0.0),
                     un * (E + p)])


def sound_speed(W, gamma=GAMMA):
    return np.sqrt(gamma * W[3] / W[0])


def rusanov(WL, WR, axis, gamma=GAMMA):
    unL = WL[1] if axis == 2 else WL[2]
    unR = WR[1] if axis == 2 else WR[2]
    a = np.maximum(np.abs(unL) + sound_speed(WL, gamma), np.abs(unR) + sound_speed(WR, gamma))
    FL, FR = physical_flux(WL, axis, gamma), physical_flux(WR, axis, gamma)
    UL, UR = conserved(WL, gamma), conserved(WR, gamma)
    return 0.5 * (FL + FR) - 0.5 * a * (UR - UL)


# ------------------------------------------------------------------ pass 5
def rhs(U, dx, dy, gamma=GAMMA):
    """L(U): minus the flux divergence, each pass over the whole grid."""
    W = primitives(U, gamma)
    out = np.zeros_like(U)
    for axis, d in ((2, dx), (1, dy)):
        s = slopes(W, axis)
        WL, WR = face_states(W, s, axis)
        F = rusanov(WL, WR, axis, gamma)           # F[..., i] is the flux at face i + 1/2
        out -= (F - np.roll(F, 1, axis=axis)) / d
    return out


# ------------------------------------------------------------------ pass 7
def max_wave(U, dx, dy, gamma=GAMMA):
    W = primitives(U, gamma)
    c = sound_speed(W, gamma)
    return float(np.max((np.abs(W[1]) + c) / dx + (np.abs(W[2]) + c) / dy))


# ------------------------------------------------------------------ pass 6
def step(U, dx, dy, cfl=0.4, dt=None, gamma=GAMMA):
    """One SSP-RK2 step; dt from the CFL condition unless given. Returns (U', dt)."""
    if dt is None:
        dt = cfl / max_wave(U, dx, dy, gamma)
    U1 = U + dt * rhs(U, dx, dy, gamma)
    U2 = 0.5 * (U + (U1 + dt * rhs(U1, dx, dy, gamma)))
    return U2, dt


def run(U, dx, dy, nsteps, cfl=0.4, gamma=GAMMA, dts=None):
    """nsteps steps; dts (optional) fixes each step's dt. Returns (U, [dt])."""
    out = []
    for k in range(nsteps):
        U, dt = step(U, dx, dy, cfl, None if dts is None else dts[k], gamma)
        out.append(dt)
    return U, out


# ------------------------------------------------------------------ exact Riemann solution
def _pressure_function(p, rho, pk, ck, gamma):
    """f_K(p) and its derivative: shock branch for p > p_K, rarefaction otherwise."""
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = np.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    r = p / pk
    f = 2.0 * ck / (gamma - 1.0) * (r ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)
    df = 1.0 / (rho * ck) * r ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(WL, WR, gamma=GAMMA):
    """Pressure and velocity between the left and right waves (u normal)."""
    rl, ul, pl = WL
    rr, ur, pr = WR
    cl, cr = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _pressure_function(p, rl, pl, cl, gamma)
        fr, dfr = _pressure_function(p, rr, pr, cr, gamma)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(1e-12, p - dp)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _pressure_function(p, rl, pl, cl, gamma)
    fr, _ = _pressure_function(p, rr, pr, cr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def exact_riemann(WL, WR, xi, gamma=GAMMA):
    """(rho, u, p) of the exact solution of the 1D Riemann problem with left
    and right states (rho, u, p) at the similarity coordinates xi = x / t."""
    rl, ul, pl = WL
    rr, ur, pr = WR
    cl, cr = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    ps, us = star_state(WL, WR, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.empty((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:   # left of the contact
            if ps > pl:   # left shock
                rs = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0)
                S = ul - cl * np.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl + (gamma - 1.0) / (2.0 * gamma))
                out[:, n] = (rl, ul, pl) if s < S else (rs, us, ps)
            else:         # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / gamma)
                cs = cl * (ps / pl) ** ((gamma - 1.0) / (2.0 * gamma))
                if s < ul - cl:
                    out[:, n] = (rl, ul, pl)
                elif s > us - cs:
                    out[:, n] = (rs, us, ps)
                else:     # inside the fan
                    u = 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * ul + s)
                    c = 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * (ul - s))
                    r = rl * (c / cl) ** (2.0 / (gamma - 1.0))
                    out[:, n] = (r, u, pl * (c / cl) ** (2.0 * gamma / (gamma - 1.0)))
        else:         # right of the contact
            if ps > pr:   # right shock
                rs = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0)
                S = ur + cr * np.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + (gamma - 1.0) / (2.0 * gamma))
                out[:, n] = (rr, ur, pr) if s > S else (rs, us, ps)
            else:         # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / gamma)
                cs = cr * (ps / pr) ** ((gamma - 1.0) / (2.0 * gamma))
                if s > ur + cr:
                    out[:, n] = (rr, ur, pr)
                elif s < us + cs:
                    out[:, n] = (rs, us, ps)
                else:
                    u = 2.0 / (gamma + 1.0) * (-cr + 0.5 * (gamma - 1.0) * ur + s)
                    c = 2.0 / (gamma + 1.0) * (cr - 0.5 * (gamma - 1.0) * (ur - s))
                    r = rr * (c / cr) ** (2.0 / (gamma - 1.0))
                    out[:, n] = (r, u, pr * (c / cr) ** (2.0 * gamma / (gamma - 1.0)))
    return out


# ------------------------------------------------------------------ workloads of the pins and tests
def isentropic_vortex(nx, ny, L=10.0, beta=5.0, u0=1.0, v0=1.0, t=0.0, gamma=GAMMA):
    """Point values at the cell centres of the isentropic vortex advected by
    the mean flow (u0, v0) for time t on the periodic square [0, L)^2, centred
    at L/2 at t = 0 (rho = p = 1 far away). Returns U (4, ny, nx)."""
    h = L / nx
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * (L / ny)
    X, Y = np.meshgrid(x, y)
    # nearest periodic image of the moving centre
    dxv = (X - (0.5 * L + u0 * t)) % L
    dyv = (Y - (0.5 * L + v0 * t)) % L
    dxv = np.where(dxv > 0.5 * L, dxv - L, dxv)
    dyv = np.where(dyv > 0.5 * L, dyv - L, dyv)
    r2 = dxv * dxv + dyv * dyv
    e = np.exp(0.5 * (1.0 - r2))
    u = u0 - beta / (2.0 * np.pi) * dyv * e
    v = v0 + beta / (2.0 * np.pi) * dxv * e
    T = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * np.pi * np.pi) * e * e
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return conserved(np.stack([rho, u, v, p]), gamma)
