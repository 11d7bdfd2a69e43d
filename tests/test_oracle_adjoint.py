"""Pins of the oracle's discrete adjoint against facts it does not compute
itself: the closed-form Jacobian of RK4 on a linear field, and central finite
differences of the (separately pinned) oracle forward."""
import numpy as np

import oracle
from paper_2004_02003_gb300 import inputs


def _R(Z):
    """RK4 stability matrix: the Jacobian of one RK4 step of x' = A x + b."""
    I = np.eye(3)
    return I + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24


def test_adjoint_seed_gradient_linear_field_closed_form():
    A = np.array([[-0.75, 1.5, 0.25], [-1.25, 0.5, -0.5], [0.375, -0.25, -1.0]])
    b = np.array([0.5, -0.25, 0.125])
    n, h, origin = (64, 64, 64), (0.25,) * 3, (-8.0,) * 3
    g = oracle.Grid.make(n, origin, h)
    field = inputs.affine_field(n, origin, h, A, b)
    rng = np.random.default_rng(4)
    x0 = rng.uniform(-0.5, 0.5, size=(40, 3))
    L, dt = 10, 0.0625
    lam_end = rng.standard_normal((40, 3))
    st, lam0, _ = oracle.vjp(g, lambda c: field, dt, x0, L, lam_end)
    assert np.all(st.exit_cycle < 0)
    M = np.linalg.matrix_power(_R(dt * A), L)        # dx_end / dx0
    assert np.max(np.abs(lam0 - lam_end @ M)) < 1e-11


def _loss(g, fields, dt, x0, L, w):
    s = oracle.State(x0)
    for c in range(L):
        oracle.cycle(g, fields[c], dt, c, s)
    return float(np.sum(w * s.x)), s


def test_adjoint_seed_gradient_matches_central_differences_on_abc():
    n, h = (32, 32, 32), (2 * np.pi / 32,) * 3
    g = oracle.Grid.make(n, (0, 0, 0), h)
    L, dt = 12, 0.02
    fields = [inputs.abc_field(n, (0, 0, 0), h, c * dt) for c in range(L)]
    rng = np.random.default_rng(5)
    x0 = rng.uniform(1.5, 2 * np.pi - 1.5, size=(24, 3))
    w = rng.standard_normal((24, 3))
    st, lam0, _ = oracle.vjp(g, lambda c: fields[c], dt, x0, L, w)
    assert np.all(st.exit_cycle < 0)
    eps = 1e-6
    fd = np.zeros_like(x0)
    for p in range(x0.shape[0]):
        for a in range(3):
            xp = x0[p:p + 1].copy(); xp[0, a] += eps
            xm = x0[p:p + 1].copy(); xm[0, a] -= eps
            lp, _ = _loss(g, fields, dt, xp, L, w[p:p + 1])
            lm, _ = _loss(g, fields, dt, xm, L, w[p:p + 1])
            fd[p, a] = (lp - lm) / (2 * eps)
    rel = np.abs(fd - lam0) / (np.abs(lam0) + 1e-3)
    assert np.median(rel) < 1e-6
    assert np.mean(rel < 1e-5) >= 0.95          # a kink crossing may spoil a few


def test_adjoint_field_gradient_matches_central_differences():
    # Non-affine (ABC) field, perturb single node components of single cycles.
    n, h = (16, 16, 16), (2 * np.pi / 16,) * 3
    g = oracle.Grid.make(n, (0, 0, 0), h)
    L, dt = 6, 0.05
    fields = [inputs.abc_field(n, (0, 0, 0), h, c * dt) for c in range(L)]
    rng = np.random.default_rng(6)
    x0 = rng.uniform(2.0, 2 * np.pi - 2.0, size=(64, 3))
    w = rng.standard_normal((64, 3))
    st, _, gF = oracle.vjp(g, lambda c: fields[c], dt, x0, L, w, want_field_grads=True)
    # pick node components with non-negligible gradient
    picks = []
    for c in range(L):
        flat = np.abs(gF[c]).ravel()
        for idx in np.argsort(flat)[-3:]:
            picks.append((c, idx))
    eps = 1e-2
    for c, idx in picks:
        fp = [f.copy() for f in fields]
        fm = [f.copy() for f in fields]
        fp[c].ravel()[idx] += eps
        fm[c].ravel()[idx] -= eps
        lp, _ = _loss(g, fp, dt, x0, L, w)
        lm, _ = _loss(g, fm, dt, x0, L, w)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - gF[c].ravel()[idx]) <= 2e-3 * abs(gF[c].ravel()[idx]) + 1e-6, (c, idx)


def test_adjoint_stops_at_the_exit_cycle():
    # Expanding linear flow u = A (x - c): a particle near a face leaves at
    # cycle e, its end is x_e = R^e applied to x0, so d end / d x0 = R^e;
    # one that stays gets R^L.
    A = 0.25 * np.eye(3) + np.array([[0.0, 0.125, 0.0], [-0.125, 0.0, 0.0], [0.0, 0.0, 0.0]])  # dyadic
    c = np.array([8.0, 8.0, 8.0])
    n, h, L, dt = (16, 16, 16), (1.0, 1.0, 1.0), 12, 0.25
    g = oracle.Grid.make(n, (0, 0, 0), h)
    field = inputs.affine_field(n, (0, 0, 0), h, A, -A @ c)
    x0 = np.array([[13.5, 8.25, 8.5], [8.5, 8.25, 8.125]])
    lam_end = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]])
    st, lam0, _ = oracle.vjp(g, lambda k: field, dt, x0, L, lam_end)
    e = st.exit_cycle
    assert 0 < e[0] < L - 1 and e[1] == -1
    R = _R(dt * A)
    assert np.max(np.abs(lam0[0] - lam_end[0] @ np.linalg.matrix_power(R, e[0]))) < 1e-11
    assert np.max(np.abs(lam0[1] - lam_end[1] @ np.linalg.matrix_power(R, L))) < 1e-11


def test_adjoint_workload_central_differences():
    # The adjoint workload's block, field and interval (64^3 ABC on
    # [0, 2 pi]^3, 200 cycles, dt 0.01) with loss = sum over the particles of
    # |end - start|^2: central differences with a step of 1e-3 cells on 64
    # start points and on 64 (cycle, node component) pairs, against the
    # discrete adjoint. The start points are random points at least 2 cells
    # from every face that stay in the block: the lattice seeds themselves sit
    # on cell corners, where the trilinear field (continuous, not
    # differentiable across faces) has only one-sided derivatives. Over 200
    # cycles some perturbed paths still cross a face at another step; the
    # error distribution is graded, not every sample.
    n, L, dt = (64, 64, 64), 200, 0.01
    hh = 2 * np.pi / 64
    g = oracle.Grid.make(n, (0, 0, 0), (hh,) * 3)
    fields = [inputs.abc_field(n, (0, 0, 0), (hh,) * 3, c * dt) for c in range(L)]
    rng = np.random.default_rng(40)
    cand = rng.uniform(2 * hh, 2 * np.pi - 2 * hh, size=(1024, 3))
    st0, _ = oracle.forward_with_history(g, lambda c: fields[c], dt, cand, L)
    x0 = cand[st0.valid == 1][:64]
    assert x0.shape[0] == 64
    st, _ = oracle.forward_with_history(g, lambda c: fields[c], dt, x0, L)
    d = st.x - x0
    # dL/dx0 = J^T 2 d - 2 d; dL/dF from the adjoint
    _, lam, gF = oracle.vjp(g, lambda c: fields[c], dt, x0, L, 2 * d, want_field_grads=True)
    grad = lam - 2 * d

    # steps of 1e-3 cells (the workload's specification): perturbed paths
    # cross faces at other steps, which bounds the agreement (measured:
    # median 7e-5, 90th percentile 3e-4, max 2e-3); steps of 1e-5 cells cross
    # almost none, and the adjoint must then agree to rounding
    for step, bounds in ((1e-3, (1e-3, 3e-3, 5e-2)), (1e-5, (1e-6, 1e-4, 5e-2))):
        eps = step * hh
        xp = np.repeat(x0, 6, axis=0)
        for a in range(3):
            xp[2 * a::6, a] += eps
            xp[2 * a + 1::6, a] -= eps
        stp, _ = oracle.forward_with_history(g, lambda c: fields[c], dt, xp, L)
        assert np.all(stp.valid == 1)
        lossp = np.sum((stp.x - xp) ** 2, axis=1).reshape(64, 3, 2)
        fd = (lossp[:, :, 0] - lossp[:, :, 1]) / (2 * eps)
        rel = (np.abs(fd - grad) / (np.abs(grad) + 1e-6 * np.abs(grad).max())).ravel()
        print(f"seed FD ({step:.0e} cells) rel err: median {np.median(rel):.1e} "
              f"p90 {np.percentile(rel, 90):.1e} max {rel.max():.1e}")
        assert np.median(rel) < bounds[0] and np.percentile(rel, 90) < bounds[1] and rel.max() < bounds[2]

    # node velocities (float32 inputs: the step actually taken is the
    # difference of the two rounded values). Measured: median 5e-9 for steps
    # of 1e-3, 3e-7 for 1e-5 (rounding of the loss difference)
    gF = np.stack(gF)
    flat = np.flatnonzero(np.abs(gF).ravel() > 1e-3 * np.abs(gF).max())
    pairs = rng.choice(flat, size=64, replace=False)
    for du, bounds in ((1e-3, (1e-6, 1e-5)), (1e-5, (1e-5, 1e-4))):
        errs = []
        for k in pairs:
            c, idx = divmod(int(k), fields[0].size)
            out, vals = [], []
            for sgn in (1.0, -1.0):
                fc = fields[c].copy()
                fc.ravel()[idx] = np.float32(float(fields[c].ravel()[idx]) + sgn * du)
                vals.append(float(fc.ravel()[idx]))
                s2, _ = oracle.forward_with_history(g, lambda cc: fc if cc == c else fields[cc], dt, x0, L)
                out.append(float(np.sum((s2.x - x0) ** 2)))
            fdv = (out[0] - out[1]) / (vals[0] - vals[1])
            errs.append(abs(fdv - gF.ravel()[k]) / abs(gF.ravel()[k]))
        errs = np.array(errs)
        print(f"field FD ({du:.0e}) rel err: median {np.median(errs):.1e} p90 {np.percentile(errs, 90):.1e} "
              f"max {errs.max():.1e}")
        assert np.median(errs) < bounds[0] and np.percentile(errs, 90) < bounds[1]
