"""The per-cell reaction step in FP64 (the path the CUDA library implements).

Order of the step (Sec. 2 states the network input (T, p, Y) and its chemical output;
the rest are this project's readings, each written out plainly):
  a0  active cells: T > T_react, listed in ascending cell index;
  a1-a4  real-fluid state of each active cell and its enthalpy h0 = h(T, p, Y) (pr_eos);
  a5  network inputs: Z-scored (T, p, BC(Y)) (network.normalise_inputs);
  a6-a7  MLP forward (network.mlp_forward);
  a8  Y' from the de-normalised outputs (network.denormalise);
  a9  T' from h(T', p, Y') = h0 by safeguarded Newton (enthalpy is conserved in the
      adiabatic, isobaric reactor the network stands in for);
  a10 write-back of T', Y' for active cells; inactive cells are left as they were.

Per-cell status bits: 1 Newton not converged, 2 no cubic root above B, 4 non-finite input
or result. A flagged cell is left as it was.
"""
from __future__ import annotations

import numpy as np

from . import network as nw
from .pr_eos import NO_ROOT, state

NOT_CONVERGED = 1
NONFINITE = 4
T_LO, T_HI = 50.0, 5000.0


def active_cells(T, T_react):
    """Indices i with T_i > T_react, ascending (a stable compaction of the cell list)."""
    return np.flatnonzero(np.asarray(T) > T_react).astype(np.int64)


def enthalpy_cp(mech, T, p, Y):
    s = state(mech, T, p, Y)
    return s["h"], s["cp"], s["status"]


def solve_T(mech, p, Y, h0, T_start, tol=1e-12, max_iter=100, return_iters=False):
    """Newton on h(T, p, Y) = h0 with slope cp, kept inside a bracket [lo, hi] that starts
    at [50, 5000] K and shrinks with the sign of h - h0 (h rises with T). Stops when the
    Newton step |dT| <= tol * T; a longer step that leaves the bracket is replaced by
    bisection."""
    T = np.clip(np.asarray(T_start, dtype=np.float64).copy(), T_LO, T_HI)
    lo = np.full_like(T, T_LO)
    hi = np.full_like(T, T_HI)
    status = np.zeros(T.shape, dtype=np.int32)
    iters = np.zeros(T.shape, dtype=np.int64)
    todo = np.ones(T.shape, dtype=bool)
    for _ in range(max_iter):
        if not todo.any():
            break
        idx = np.flatnonzero(todo)
        h, cp, st = enthalpy_cp(mech, T[idx], p[idx], Y[:, idx])
        bad = st != 0
        status[idx[bad]] |= st[bad]
        f = h - h0[idx]
        hi[idx] = np.where(f > 0.0, np.minimum(hi[idx], T[idx]), hi[idx])
        lo[idx] = np.where(f <= 0.0, np.maximum(lo[idx], T[idx]), lo[idx])
        with np.errstate(divide="ignore", invalid="ignore"):
            Tn = T[idx] - f / cp
        # a step within tolerance has converged; only a longer step that leaves the
        # bracket (or is not finite) is replaced by bisection
        done = np.isfinite(Tn) & (np.abs(Tn - T[idx]) <= tol * T[idx])
        out = ~done & (~np.isfinite(Tn) | (Tn <= lo[idx]) | (Tn >= hi[idx]))
        Tn = np.where(out, 0.5 * (lo[idx] + hi[idx]), Tn)
        T[idx] = Tn
        iters[idx] += 1
        finished = done | bad
        todo[idx[finished]] = False
    status[todo] |= NOT_CONVERGED
    return (T, status, iters) if return_iters else (T, status)


def chem_step(mech, net, T, p, Y, dt, T_react=600.0, newton_tol=1e-12, max_iter=100,
              return_parts=False):
    """One reaction step of every cell. T [N], p [N], Y [n, N] are not modified; returns
    (T_new, Y_new, status) and, if asked, the intermediate arrays of the active cells."""
    if abs(dt - net.dt) > 1e-12 * abs(net.dt):
        raise ValueError("dt differs from the time step the network was built for")
    T = np.asarray(T, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    N = T.shape[0]
    status = np.where(np.isfinite(T), 0, NONFINITE).astype(np.int32)
    idx = active_cells(T, T_react)
    Ta, pa, Ya = T[idx], p[idx], Y[:, idx]
    finite = np.isfinite(pa) & np.all(np.isfinite(Ya), axis=0) & (pa > 0.0)
    st0 = state(mech, Ta, pa, Ya)                       # a1-a4
    h0 = st0["h"]
    x = nw.normalise_inputs(net, Ta, pa, Ya)            # a5
    O = nw.mlp_forward(net, x)                          # a6-a7
    Yn = nw.denormalise(net, Ya, O)                     # a8
    Tn, st = solve_T(mech, pa, Yn, h0, Ta, newton_tol, max_iter)   # a9
    st = st | st0["status"]
    st = np.where(finite, st, NONFINITE)
    ok = (st == 0) & np.isfinite(Tn) & np.all(np.isfinite(Yn), axis=0)
    st = np.where(ok | (st != 0), st, NONFINITE)
    T_out = T.copy()
    Y_out = Y.copy()
    T_out[idx[ok]] = Tn[ok]                             # a10
    Y_out[:, idx[ok]] = Yn[:, ok]
    status[idx] = st
    if return_parts:
        return T_out, Y_out, status, dict(idx=idx, h0=h0, state=st0, x=x, O=O, Y_new=Yn, T_new=Tn)
    return T_out, Y_out, status


def real_fluid_props(mech, T, p, Y):
    """(rho, h, cp, Z) of every cell, with h in J/kg and cp in J/(kg K)."""
    s = state(mech, T, p, Y)
    return s["rho"], s["h"], s["cp"], s["Z"]


def chem_source(mech, net, T, p, Y, dt, T_react=600.0, newton_tol=1e-12, max_iter=100):
    """Chemical source terms of the step for a flow solver (the network supplies the chemical
    change of each cell, Sec. 2): omega_k = rho (Y'_k - Y_k) / dt in kg/(m^3 s), rho the
    real-fluid density at the cell's state (T, p, Y), with (T', Y') from chem_step. Cells
    that do not react or are flagged get omega = 0 and T' = T. Returns (omega [n, N], T', status)."""
    T = np.asarray(T, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Tn, Yn, status = chem_step(mech, net, T, p, Y, dt, T_react, newton_tol, max_iter)
    omega = np.zeros_like(Y)
    idx = active_cells(T, T_react)
    idx = idx[status[idx] == 0]
    if idx.size:
        rho = state(mech, T[idx], p[idx], Y[:, idx])["rho"]
        omega[:, idx] = rho[None, :] * (Yn[:, idx] - Y[:, idx]) / dt
    return omega, Tn, status


def chem_step_vjp(mech, net, T, p, Y, gT, gY, T_react=600.0, **fd):
    """Reverse-mode product of the reaction step: given cotangents gT [N] and gY [n, N] of the
    step's outputs (T', Y'), the cotangents of its inputs (T, Y) with p fixed,
        g_v = gT dT'/dv + sum_k gY_k dY'_k/dv,   v = (T, Y_1..Y_n),
    from chem_step_jacobian_fd (keyword arguments go to it) with Y'_k = Y_k + dY_k. Cells that
    do not react (T <= T_react, or a non-finite T) are left as they were by the step, so their
    cotangents pass through. Returns (g_T [N], g_Y [n, N]); entries whose Jacobian column is
    NaN (species below the difference floor) are NaN. The paper prints no derivative of the
    step (its networks are trained offline); this is the transpose of the step's Jacobian,
    applied to the cotangents, by definition of the chain rule."""
    T = np.asarray(T, dtype=np.float64)
    gT = np.asarray(gT, dtype=np.float64)
    gY = np.asarray(gY, dtype=np.float64)
    J, dTn = chem_step_jacobian_fd(mech, net, T, p, Y, **fd)
    n, N = gY.shape
    g = np.empty((N, n + 1))
    for c in range(N):
        dYp = J[c] + np.hstack([np.zeros((n, 1)), np.eye(n)])   # dY'_k/dv_t
        g[c] = gT[c] * dTn[c] + gY[:, c] @ dYp
    passive = ~(T > T_react)
    g[passive, 0] = gT[passive]
    g[passive, 1:] = gY[:, passive].T
    return g[:, 0].copy(), g[:, 1:].T.copy()


__all__ = ["active_cells", "solve_T", "chem_step", "chem_source", "real_fluid_props", "chem_step_vjp",
           "NOT_CONVERGED", "NONFINITE", "NO_ROOT"]


def chem_step_jacobian_fd(mech, net, T, p, Y, dT_rel=1e-6, dY_rel=1e-5, dY_min=1e-6):
    """Central finite differences of the reaction step of each cell (treated as active):
    J_dY [N, n, n+1] = d(Y'_k - Y_k) / d(T, Y_1..Y_n) and dTn [N, n+1] = dT'/d(T, Y_1..Y_n),
    with p fixed and the Y_j perturbed independently (no renormalisation of the input).
    Steps: T by dT_rel * T, Y_j by dY_rel * Y_j; species with Y_j < dY_min get NaN columns
    (the Box-Cox transform is not differentiable at 0, so a difference there means nothing)."""
    T = np.asarray(T, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n, N = Y.shape
    J = np.full((N, n, n + 1), np.nan)
    dTn = np.full((N, n + 1), np.nan)

    def run(Tx, Yx):
        To, Yo, st = chem_step(mech, net, Tx, p, Yx, net.dt, T_react=-1.0)
        return To, Yo - Yx, st

    h = dT_rel * T
    Tp, dYp, sp = run(T + h, Y)
    Tm, dYm, sm = run(T - h, Y)
    J[:, :, 0] = ((dYp - dYm) / (2 * h)).T
    dTn[:, 0] = (Tp - Tm) / (2 * h)
    for j in range(n):
        ok = Y[j] >= dY_min
        hj = np.where(ok, dY_rel * Y[j], 0.0)
        Yp = Y.copy(); Yp[j] += hj
        Ym = Y.copy(); Ym[j] -= hj
        Tp, dYp, _ = run(T, Yp)
        Tm, dYm, _ = run(T, Ym)
        with np.errstate(invalid="ignore", divide="ignore"):
            col = ((dYp - dYm) / (2 * hj)).T
            tcol = (Tp - Tm) / (2 * hj)
        J[:, :, 1 + j] = np.where(ok[:, None], col, np.nan)
        dTn[:, 1 + j] = np.where(ok, tcol, np.nan)
    return J, dTn
