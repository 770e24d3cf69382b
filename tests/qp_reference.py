"""Independent references used to pin the oracle (numpy / scipy only; imports nothing from oracle/).

* ``original_qp``      -- the MPC problem of Sec. II (eqn. for the LTV MPC) as an explicit dense QP in
                          y = (u_0, x_1, ..., u_{N-1}, x_N), plus the optional input-increment weight.
* ``kkt_enumerate``    -- brute-force active-set enumeration of that QP (every variable free / at
                          its lower bound / at its upper bound), keeping the KKT point.
* ``equality_qp``      -- the same QP with all bounds dropped (or some variables fixed), solved by
                          one dense KKT linear solve.
* ``velocity_FGh``     -- the velocity-form splitting (Theorem 2 and the problem it reformulates)
                          written as the generic constrained form min f(p) + g(q), Fp + Gq = h.
* ``generic_admm_step``-- one scaled-form ADMM pass on that generic form (Boyd et al.): a dense
                          least-squares solve for p, a bounded least-squares solve for q
                          (scipy lsq_linear, BVLS), the dual update and the residual
                          c = rho ||s+ - s||^2 + rho ||G (q+ - q)||^2.
* ``generic_admm_step_set``, ``solve_set_qp`` -- the same with the inputs in a non-box convex set
                          (l2 ball, l1 ball, halfspace, second-order cone), by SLSQP.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.optimize import lsq_linear


def _stage(inst, key, k):
    a = np.asarray(inst[key], dtype=np.float64)
    return a if inst.get("lti", False) else a[k]


def _ref(inst):
    N, n = inst["N"], inst["nx"] + inst["nu"]
    return np.broadcast_to(np.asarray(inst["ref"], np.float64), (N, n))


# ---------------------------------------------------------------------------------------------
# The MPC problem as an explicit QP in the original variables.
# ---------------------------------------------------------------------------------------------

def original_qp(inst):
    """Returns (P, c, Aeq, beq, lb, ub, idx) for  min 1/2 y'Py + c'y  s.t. Aeq y = beq, lb <= y <= ub.
    idx(k, 'u'|'x') gives the slice of u_k or x_{k+1} in y."""
    nx, nu, N = inst["nx"], inst["nu"], inst["N"]
    blk = nx + nu
    dim = N * blk
    ref = _ref(inst)

    def idx(k, which):
        o = k * blk
        return slice(o, o + nu) if which == "u" else slice(o + nu, o + blk)

    P = np.zeros((dim, dim))
    c = np.zeros(dim)
    q, r = np.asarray(inst["q"], float), np.asarray(inst["r"], float)
    rdu = None if inst.get("rdu") is None else np.asarray(inst["rdu"], float)
    uprev = np.zeros(nu) if inst.get("u_prev") is None else np.asarray(inst["u_prev"], float)
    for k in range(N):
        sx, su = idx(k, "x"), idx(k, "u")
        # 1/2 ||x_{k+1} - r_x||_Q^2 + 1/2 ||u_k - r_u||_R^2
        P[sx, sx] += np.diag(q)
        c[sx] -= q * ref[k, :nx]
        P[su, su] += np.diag(r)
        c[su] -= r * ref[k, nx:]
        if rdu is not None:
            # 1/2 (u_k - u_{k-1})' W (u_k - u_{k-1}), u_{-1} = u_prev
            P[su, su] += np.diag(rdu)
            if k > 0:
                sp = idx(k - 1, "u")
                P[sp, sp] += np.diag(rdu)
                P[su, sp] -= np.diag(rdu)
                P[sp, su] -= np.diag(rdu)
            else:
                c[su] -= rdu * uprev
    Aeq = np.zeros((N * nx, dim))
    beq = np.zeros(N * nx)
    x0 = np.asarray(inst["x0"], float)
    for k in range(N):
        A, B, e = _stage(inst, "A", k), _stage(inst, "B", k), _stage(inst, "e", k)
        rows = slice(k * nx, (k + 1) * nx)
        # x_{k+1} - A_k x_k - B_k u_k = e_k
        Aeq[rows, idx(k, "x")] = np.eye(nx)
        Aeq[rows, idx(k, "u")] = -B
        if k == 0:
            beq[rows] = e + A @ x0
        else:
            Aeq[rows, idx(k - 1, "x")] = -A
            beq[rows] = e
    lb = np.zeros(dim)
    ub = np.zeros(dim)
    for k in range(N):
        lb[idx(k, "u")], ub[idx(k, "u")] = inst["umin"], inst["umax"]
        lb[idx(k, "x")], ub[idx(k, "x")] = inst["xmin"], inst["xmax"]
    return P, c, Aeq, beq, lb, ub, idx


def equality_qp(P, c, Aeq, beq, fixed=None):
    """Minimise 1/2 y'Py + c'y s.t. Aeq y = beq and y_i = v_i for (i, v) in ``fixed``.
    Returns (y, g) with g = P y + c + Aeq' nu the reduced gradient."""
    dim = P.shape[0]
    fixed = fixed or []
    m = Aeq.shape[0]
    E = np.zeros((len(fixed), dim))
    bf = np.zeros(len(fixed))
    for j, (i, v) in enumerate(fixed):
        E[j, i] = 1.0
        bf[j] = v
    C = np.vstack([Aeq, E])
    K = np.block([[P, C.T], [C, np.zeros((C.shape[0], C.shape[0]))]])
    rhs = np.concatenate([-c, beq, bf])
    sol = np.linalg.lstsq(K, rhs, rcond=None)[0] if np.linalg.matrix_rank(K) < K.shape[0] \
        else np.linalg.solve(K, rhs)
    y = sol[:dim]
    nu = sol[dim:dim + m]
    g = P @ y + c + Aeq.T @ nu
    return y, g


def kkt_enumerate(P, c, Aeq, beq, lb, ub, tol=1e-9):
    """Brute force over every assignment {free, at lb, at ub} of the bounded variables; returns the
    unique primal-feasible assignment with correctly signed bound multipliers."""
    dim = P.shape[0]
    bounded = [i for i in range(dim) if np.isfinite(lb[i]) or np.isfinite(ub[i])]
    best = []
    for states in itertools.product((0, 1, 2), repeat=len(bounded)):
        fixed = []
        ok = True
        for i, s in zip(bounded, states):
            if s == 1:
                if not np.isfinite(lb[i]):
                    ok = False; break
                fixed.append((i, lb[i]))
            elif s == 2:
                if not np.isfinite(ub[i]):
                    ok = False; break
                fixed.append((i, ub[i]))
        if not ok:
            continue
        y, g = equality_qp(P, c, Aeq, beq, fixed)
        if np.any(y < lb - tol) or np.any(y > ub + tol):
            continue
        if np.abs(Aeq @ y - beq).max() > 1e-8:
            continue
        good = True
        for i, s in zip(bounded, states):
            if s == 1 and g[i] < -tol:
                good = False; break
            if s == 2 and g[i] > tol:
                good = False; break
            if s == 0 and abs(g[i]) > 1e-7:
                good = False; break
        if good:
            best.append((y, states))
    return best


# ---------------------------------------------------------------------------------------------
# The velocity-form splitting in the generic form  min f(p) + g(q), F p + G q = h.
# ---------------------------------------------------------------------------------------------

def velocity_FGh(inst):
    """p = (du_0..du_{N-1}, xbar_1..xbar_N), q = (v_0..v_{N-1}, z_1..z_N),
    s = (theta_0..theta_{N-1}, beta_0..beta_{N-1}, lambda_0..lambda_{N-1}).
    Constraint blocks (Theorem 2 problem):
      theta_k : xbar_{k+1} - z_{k+1} = 0
      beta_k  : Bbar_k du_k - v_k = 0
      lambda_k: z_{k+1} - Abar_k xbar_k - v_k - ebar_k = 0, xbar_0 = (x0, u_prev) given.
    Returns dict(F, G, h, Pf, cf, lb, ub, sizes) with f(p) = 1/2 p'Pf p + cf'p and the box on z."""
    nx, nu, N = inst["nx"], inst["nu"], inst["N"]
    n = nx + nu
    dp = N * nu + N * n
    dq = 2 * N * n
    ds = 3 * N * n
    F = np.zeros((ds, dp))
    G = np.zeros((ds, dq))
    h = np.zeros(ds)
    du = lambda k: slice(k * nu, (k + 1) * nu)
    xb = lambda k1: slice(N * nu + (k1 - 1) * n, N * nu + k1 * n)  # xbar_{k1}, k1 = 1..N
    v = lambda k: slice(k * n, (k + 1) * n)
    z = lambda k1: slice(N * n + (k1 - 1) * n, N * n + k1 * n)     # z_{k1}, k1 = 1..N
    th = lambda k: slice(k * n, (k + 1) * n)
    be = lambda k: slice(N * n + k * n, N * n + (k + 1) * n)
    la = lambda k: slice(2 * N * n + k * n, 2 * N * n + (k + 1) * n)
    uprev = np.zeros(nu) if inst.get("u_prev") is None else np.asarray(inst["u_prev"], float)
    xbar0 = np.concatenate([np.asarray(inst["x0"], float), uprev])
    I = np.eye(n)
    for k in range(N):
        A, B, e = _stage(inst, "A", k), _stage(inst, "B", k), _stage(inst, "e", k)
        Abar = np.block([[A, B], [np.zeros((nu, nx)), np.eye(nu)]])
        Bbar = np.vstack([B, np.eye(nu)])
        ebar = np.concatenate([e, np.zeros(nu)])
        F[th(k), xb(k + 1)] = I
        G[th(k), z(k + 1)] = -I
        F[be(k), du(k)] = Bbar
        G[be(k), v(k)] = -I
        G[la(k), z(k + 1)] = I
        G[la(k), v(k)] = -I
        if k == 0:
            h[la(k)] = ebar + Abar @ xbar0
        else:
            F[la(k), xb(k)] = -Abar
            h[la(k)] = ebar
    Pf = np.zeros((dp, dp))
    cf = np.zeros(dp)
    qbar = np.concatenate([np.asarray(inst["q"], float), np.asarray(inst["r"], float)])
    ref = _ref(inst)
    for k in range(N):
        Pf[xb(k + 1), xb(k + 1)] = np.diag(qbar)
        cf[xb(k + 1)] = -qbar * ref[k]
        if inst.get("rdu") is not None:
            Pf[du(k), du(k)] = np.diag(np.asarray(inst["rdu"], float))
    lo = np.concatenate([inst["xmin"], inst["umin"]]).astype(float)
    hi = np.concatenate([inst["xmax"], inst["umax"]]).astype(float)
    lb = np.concatenate([-np.inf * np.ones(N * n), np.tile(lo, N)])
    ub = np.concatenate([np.inf * np.ones(N * n), np.tile(hi, N)])
    return dict(F=F, G=G, h=h, Pf=Pf, cf=cf, lb=lb, ub=ub,
                slices=dict(du=du, xb=xb, v=v, z=z, th=th, be=be, la=la))


def generic_admm_step(sys_, rho, qhat, shat):
    """One scaled-form ADMM pass: p+ = argmin f(p) + rho/2 ||Fp + G qhat - h + shat||^2,
    q+ = argmin g(q) + rho/2 ||F p+ + G q - h + shat||^2 (g = box indicator on z),
    s+ = shat + F p+ + G q+ - h, c = rho ||s+ - shat||^2 + rho ||G (q+ - qhat)||^2."""
    F, G, h, Pf, cf = sys_["F"], sys_["G"], sys_["h"], sys_["Pf"], sys_["cf"]
    lhs = Pf + rho * F.T @ F
    rhs = -cf - rho * F.T @ (G @ qhat - h + shat)
    p = np.linalg.solve(lhs, rhs)
    b = h - F @ p - shat
    res = lsq_linear(G, b, bounds=(sys_["lb"], sys_["ub"]), method="bvls", tol=1e-15,
                     max_iter=10000)
    q = res.x
    s = shat + F @ p + G @ q - h
    c = rho * np.sum((s - shat) ** 2) + rho * np.sum((G @ (q - qhat)) ** 2)
    return p, q, s, c


# ---------------------------------------------------------------------------------------------
# Non-box input sets (the remark after Theorem 1): the same references with u_k in a convex set,
# solved by a general nonlinear-programming routine (scipy SLSQP) instead of a closed form.
# ---------------------------------------------------------------------------------------------

def set_constraints(inst, u_slices):
    """scipy constraint dicts keeping every u-slice of the variable vector in the instance's
    input set. Smooth descriptions: ||u||^2 <= r^2; the l1 ball as the 2^nu inequalities
    s'u <= r over sign vectors s; a'u <= r; t >= 0 and t^2 >= ||s||^2 for the cone."""
    us = inst["uset"]
    kind, r = us["kind"], float(us.get("r", 0.0))
    nu = inst["nu"]
    cons = []
    for sl in u_slices:
        if kind == 1:
            cons.append(dict(type="ineq", fun=lambda y, sl=sl: r * r - np.sum(y[sl] ** 2),
                             jac=lambda y, sl=sl: _grad_at(y, sl, -2.0 * y[sl])))
        elif kind == 2:
            for signs in itertools.product((-1.0, 1.0), repeat=nu):
                sv = np.array(signs)
                cons.append(dict(type="ineq", fun=lambda y, sl=sl, sv=sv: r - sv @ y[sl],
                                 jac=lambda y, sl=sl, sv=sv: _grad_at(y, sl, -sv)))
        elif kind == 3:
            a = np.asarray(us["a"], float)
            cons.append(dict(type="ineq", fun=lambda y, sl=sl: r - a @ y[sl],
                             jac=lambda y, sl=sl: _grad_at(y, sl, -a)))
        elif kind == 4:
            def cone(y, sl=sl):
                u = y[sl]
                return u[0] * u[0] - np.sum(u[1:] ** 2)

            def cone_jac(y, sl=sl):
                u = y[sl]
                return _grad_at(y, sl, np.concatenate([[2.0 * u[0]], -2.0 * u[1:]]))
            cons.append(dict(type="ineq", fun=cone, jac=cone_jac))
            cons.append(dict(type="ineq", fun=lambda y, sl=sl: y[sl][0],
                             jac=lambda y, sl=sl: _grad_at(y, sl, np.eye(nu)[0])))
        else:
            raise ValueError("not a non-box set")
    return cons


def _grad_at(y, sl, g):
    out = np.zeros_like(y)
    out[sl] = g
    return out


def _slsqp(fun, jac, x0, bounds, cons):
    from scipy.optimize import minimize
    res = minimize(fun, x0, jac=jac, method="SLSQP", bounds=bounds, constraints=cons,
                   options=dict(ftol=1e-16, maxiter=2000))
    return res.x


def generic_admm_step_set(sys_, rho, qhat, shat, inst):
    """generic_admm_step with g = indicator of {z_{k+1} = (x, u): x in the box, u in U}: the
    q-update is the same constrained least-squares problem, solved by SLSQP."""
    F, G, h, Pf, cf = sys_["F"], sys_["G"], sys_["h"], sys_["Pf"], sys_["cf"]
    lhs = Pf + rho * F.T @ F
    rhs = -cf - rho * F.T @ (G @ qhat - h + shat)
    p = np.linalg.solve(lhs, rhs)
    b = h - F @ p - shat
    nx, nu, N = inst["nx"], inst["nu"], inst["N"]
    n = nx + nu
    bounds = []
    for i in range(2 * N * n):
        lo, hi = sys_["lb"][i], sys_["ub"][i]
        in_z_u = i >= N * n and (i - N * n) % n >= nx
        bounds.append((None, None) if in_z_u else
                      (None if not np.isfinite(lo) else lo, None if not np.isfinite(hi) else hi))
    u_sl = [slice(N * n + k * n + nx, N * n + (k + 1) * n) for k in range(N)]
    GtG, Gtb = G.T @ G, G.T @ b
    q0 = np.linalg.lstsq(G, b, rcond=None)[0]
    q = _slsqp(lambda y: 0.5 * y @ GtG @ y - Gtb @ y, lambda y: GtG @ y - Gtb, q0, bounds,
               set_constraints(inst, u_sl))
    s = shat + F @ p + G @ q - h
    c = rho * np.sum((s - shat) ** 2) + rho * np.sum((G @ (q - qhat)) ** 2)
    return p, q, s, c


def solve_set_qp(inst):
    """The MPC problem of Sec. II with u_k in the instance's input set (and the state box), in
    y = (u_0, x_1, ..., u_{N-1}, x_N), solved by SLSQP."""
    P, c, Aeq, beq, lb, ub, idx = original_qp(inst)
    N = inst["N"]
    bounds = []
    dim = len(c)
    u_idx = np.zeros(dim, bool)
    for k in range(N):
        u_idx[idx(k, "u")] = True
    for i in range(dim):
        if u_idx[i]:
            bounds.append((None, None))
        else:
            bounds.append((None if not np.isfinite(lb[i]) else lb[i],
                           None if not np.isfinite(ub[i]) else ub[i]))
    cons = set_constraints(inst, [idx(k, "u") for k in range(N)])
    cons.append(dict(type="eq", fun=lambda y: Aeq @ y - beq, jac=lambda y: Aeq))
    y0 = equality_qp(P, c, Aeq, beq)[0]
    y = _slsqp(lambda y: 0.5 * y @ P @ y + c @ y, lambda y: P @ y + c, y0, bounds, cons)
    return y, idx
