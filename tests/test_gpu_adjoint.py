"""GPU adjoint (libbto tape) against closed forms and the FP64 oracle adjoint.

Tolerance for the FP32 adjoint against the FP64 oracle. Each RK4 step costs
about a hundred FP32 operations per component (relative rounding 6e-8 each),
and 200 steps chain them through Jacobians of norm up to ~10, so relative
errors up to ~1e-4 are expected. The trilinear field is only continuous
across cell faces: its gradient jumps there, so a particle whose FP32 path
puts a sample point (a step's start or one of its stage points) in another
cell than the FP64 path picks up an O(1) relative change of that stage's
Jacobian. Such particles are the ones whose FP64 sample points come within
CELL_EPS of a cell face, where the FP32 and FP64 paths (apart by ~1e-5
cells at most) can straddle the face, together with those whose exit cycles
differ. They are excluded, counted and the count bounded (5% of the
particles for the seed gradients, 12% of the valid ones, which sample more
cycles, for the Jacobian); every other particle is held to a maximum
relative error of 2e-3 (no percentile), 3x the largest measured.
"""
import numpy as np
import pytest

import oracle
from paper_2004_02003_gb300 import adjoint, bto, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    from paper_2004_02003_gb300 import build
    build.build()
    bto.load()
    import torch
    torch.cuda.set_device(0)


def _R(Z):
    I = np.eye(3)
    return I + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24


def _fields_dev(fields):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.stack(fields))).cuda()


def _tape_vjp(n, origin, h, seeds, fields, dt, g, K=4, want_fields=False):
    import torch
    tape = adjoint.Tape(n, origin, h, seeds.shape[0], len(fields), K)
    s = torch.from_numpy(seeds.astype(np.float32)).cuda().requires_grad_(True)
    F = _fields_dev(fields).requires_grad_(want_fields)
    ends, valid, exit_cycle = adjoint.flow_map(s, F, tape, dt)
    (ends * torch.from_numpy(g.astype(np.float32)).cuda()).sum().backward()
    out = (s.grad.cpu().numpy().astype(np.float64), ends.detach().cpu().numpy(), valid.cpu().numpy(),
           exit_cycle.cpu().numpy(), F.grad.cpu().numpy() if want_fields else None)
    tape.close()
    return out


def test_linear_field_vjp_equals_rk4_matrix_power():
    A = np.array([[-0.75, 1.5, 0.25], [-1.25, 0.5, -0.5], [0.375, -0.25, -1.0]])
    b = np.array([0.5, -0.25, 0.125])
    n, h, origin, L, dt = (64, 64, 64), (0.25,) * 3, (-8.0,) * 3, 10, 0.0625
    field = inputs.affine_field(n, origin, h, A, b)
    rng = np.random.default_rng(4)
    x0 = rng.uniform(-0.5, 0.5, size=(300, 3))
    g = rng.standard_normal((300, 3))
    grad, ends, valid, _, _ = _tape_vjp(n, origin, h, x0, [field] * L, dt, g)
    assert np.all(valid == 1)
    want = g @ np.linalg.matrix_power(_R(dt * A), L)
    assert np.max(np.abs(grad - want)) / np.max(np.abs(want)) < 2e-5


def test_gradient_stops_at_exit_cycle():
    A = 0.25 * np.eye(3) + np.array([[0.0, 0.125, 0.0], [-0.125, 0.0, 0.0], [0.0, 0.0, 0.0]])
    c = np.array([8.0, 8.0, 8.0])
    n, h, L, dt = (16, 16, 16), (1.0, 1.0, 1.0), 12, 0.25
    field = inputs.affine_field(n, (0, 0, 0), h, A, -A @ c)
    x0 = np.array([[13.5, 8.25, 8.5], [8.5, 8.25, 8.125], [20.0, 1.0, 1.0]])   # the last starts outside
    g = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0], [7.0, 8.0, 9.0]])
    grad, ends, valid, e, _ = _tape_vjp(n, (0, 0, 0), h, x0, [field] * L, dt, g, K=5)
    assert 0 < e[0] < L - 1 and e[1] == -1 and e[2] == 0
    R = _R(dt * A)
    assert np.allclose(grad[0], g[0] @ np.linalg.matrix_power(R, e[0]), rtol=2e-5)
    assert np.allclose(grad[1], g[1] @ np.linalg.matrix_power(R, L), rtol=2e-5)
    assert np.allclose(grad[2], g[2]) and np.allclose(ends[2], x0[2])


def test_checkpoint_interval_does_not_change_gradients():
    n, h, L, dt = (24, 24, 24), (2 * np.pi / 24,) * 3, 37, 0.02
    fields = [inputs.abc_field(n, (0, 0, 0), h, c * dt) for c in range(L)]
    rng = np.random.default_rng(8)
    x0 = rng.uniform(0.5, 2 * np.pi - 0.5, size=(2000, 3))
    g = rng.standard_normal((2000, 3))
    outs = [_tape_vjp(n, (0, 0, 0), h, x0, fields, dt, g, K=K, want_fields=True) for K in (1, 5, 16, 37)]
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0])
        assert np.array_equal(o[3], outs[0][3])
        assert np.allclose(o[4], outs[0][4], rtol=1e-5, atol=1e-6)   # atomics: order differs


# ----------------------------------------------------------------------------
# Adjoint workload: 64^3 block, ABC on its natural period [0, 2 pi]^3, 32^3
# seeds (stride 2), 200 cycles, dt = 0.01, checkpoints every 16 cycles.
# The oracle runs on 4096 of the seeds (particles are independent), the GPU on
# all of them and, for the field gradients, on the same 4096.
# ----------------------------------------------------------------------------
N4, L4, DT4, S4 = (64, 64, 64), 200, 0.01, 2
H4 = (2 * np.pi / 64,) * 3
# Maximum errors on every particle kept (see the module docstring; measured
# on GB300: seed gradients 6.1e-4)
SEED_GRAD_MAX_REL = 2e-3
JAC_MAX_REL = 2e-3
FTLE_MAX_ABS = 1e-3


@pytest.fixture(scope="module")
def adj_case():
    fields = [inputs.abc_field(N4, (0, 0, 0), H4, c * DT4) for c in range(L4)]
    g = oracle.Grid.make(N4, (0, 0, 0), H4)
    seeds = oracle.seeds(g, S4)
    rng = np.random.default_rng(44)
    ids = np.sort(rng.choice(seeds.shape[0], size=4096, replace=False))
    return fields, g, seeds, ids


def _loss_grad_upstream(ends, seeds, valid):
    return 2.0 * (ends - seeds) * valid[:, None]


# Sample points closer than this to a cell face (cells) may sit in another
# cell on the FP32 path. The FP32 and FP64 end positions of this workload
# differ by 2.6e-5 cells at the median (1.4e-4 at the 99th percentile), so
# a point within 1e-5 cells of a face is the one likely to straddle it.
CELL_EPS = 1e-5


def _cell_face_margin(g, fields, dt, xs, exit_cycle, h, cycles):
    """Smallest distance, in cells, from any sample point of each particle's
    FP64 oracle path (the step start and the stage points p2, p3, p4 of
    every cycle in which it is alive) to the nearest cell face plane. The
    start of the first cycle is left out: it is the seed, held exactly on
    both sides (a lattice node, on a cell corner), so both take the same
    cell there."""
    h = np.asarray(h, dtype=np.float64)
    org = np.asarray(g.origin, dtype=np.float64) if hasattr(g, "origin") else np.zeros(3)
    m = np.full(xs[0].shape[0], np.inf)
    for c in range(cycles):
        alive = (exit_cycle < 0) | (exit_cycle >= c)
        if not alive.any():
            break
        x = xs[c][alive]
        F = fields[c]
        k1 = oracle.sample(g, F, x)
        p2 = x + 0.5 * dt * k1
        k2 = oracle.sample(g, F, p2)
        p3 = x + 0.5 * dt * k2
        k3 = oracle.sample(g, F, p3)
        p4 = x + dt * k3
        for q in ((x, p2, p3, p4) if c > 0 else (p2, p3, p4)):
            xi = (q - org) / h
            d = np.abs(xi - np.round(xi)).min(axis=1)
            m[alive] = np.minimum(m[alive], d)
    return m


def test_adjoint_workload_seed_and_field_gradients_vs_oracle(adj_case):
    fields, g, seeds, ids = adj_case
    sub = seeds[ids]
    # oracle: forward to fix the loss's upstream gradient, then the adjoint
    st_o, _ = oracle.forward_with_history(g, lambda c: fields[c], DT4, sub, L4)
    up = _loss_grad_upstream(st_o.x, sub, st_o.valid)
    _, lam_o, gF_o = oracle.vjp(g, lambda c: fields[c], DT4, sub, L4, up, want_field_grads=True)
    grad_g, ends_g, valid_g, exit_g, gF_g = _tape_vjp(N4, (0, 0, 0), H4, sub, fields, DT4, up, K=16,
                                                       want_fields=True)
    assert 0.1 < st_o.valid.mean() < 0.6
    _, xs = oracle.forward_with_history(g, lambda c: fields[c], DT4, sub, L4)
    margin = _cell_face_margin(g, fields, DT4, xs, st_o.exit_cycle, H4, L4)
    keep = (exit_g == st_o.exit_cycle) & (margin >= CELL_EPS)
    excluded = int((~keep).sum())
    # seed gradients (J^T up): per-particle error relative to the gradient's size
    ref = lam_o[keep]
    err = np.linalg.norm(grad_g[keep] - ref, axis=1) / (np.linalg.norm(ref, axis=1) + 1e-6)
    live = np.linalg.norm(ref, axis=1) > 0
    print("seed-grad: %d of %d excluded (exit cycle or a sample point within %.0e cells of a cell face); "
          "rel err median %.2e max %.2e" % (excluded, len(sub), CELL_EPS, np.median(err[live]), err[live].max()))
    assert excluded <= 0.05 * len(sub)
    assert err[live].max() < SEED_GRAD_MAX_REL
    # field gradients at 64 random (cycle, node component) pairs with support
    rng = np.random.default_rng(45)
    gF_o = np.stack(gF_o)
    nz = np.flatnonzero(np.abs(gF_o) > 1e-3 * np.abs(gF_o).max())
    pick = rng.choice(nz, size=64, replace=False)
    a, b = gF_g.ravel()[pick], gF_o.ravel()[pick]
    ferr = np.abs(a - b) / (np.abs(b) + 1e-3 * np.abs(gF_o).max())
    print("field-grad rel err: median %.2e max %.2e" % (np.median(ferr), ferr.max()))
    assert np.median(ferr) < 1e-4 and ferr.max() < 2e-3


def test_adjoint_workload_jacobian_and_ftle(adj_case):
    import torch
    fields, g, seeds, ids = adj_case
    tape = adjoint.Tape(N4, (0, 0, 0), H4, seeds.shape[0], L4, 16)
    s = torch.from_numpy(seeds.astype(np.float32)).cuda()
    ends, valid, J, f = adjoint.ftle(tape, s, _fields_dev(fields), DT4)
    tape.close()
    J = J.cpu().numpy().astype(np.float64)[ids]
    f = f.cpu().numpy()[ids]
    v = valid.cpu().numpy()[ids]
    sub = seeds[ids]
    Jo = np.zeros((len(ids), 3, 3))
    for a in range(3):
        e = np.zeros((len(ids), 3)); e[:, a] = 1.0
        st, lam, _ = oracle.vjp(g, lambda c: fields[c], DT4, sub, L4, e)
        Jo[:, a, :] = lam
    _, xs = oracle.forward_with_history(g, lambda c: fields[c], DT4, sub, L4)
    margin = _cell_face_margin(g, fields, DT4, xs, st.exit_cycle, H4, L4)
    both = (v == 1) & (st.valid == 1)
    ok = both & (margin >= CELL_EPS)
    excluded = int((both & ~ok).sum())
    assert ok.sum() > 500 and excluded <= 0.12 * both.sum()
    rel = np.linalg.norm((J - Jo)[ok], axis=(1, 2)) / np.linalg.norm(Jo[ok], axis=(1, 2))
    # FTLE from the oracle Jacobian, by numpy's symmetric eigensolver
    lmax = np.linalg.eigvalsh(np.einsum("pki,pkj->pij", Jo[ok], Jo[ok]))[:, -1]
    f_o = 0.5 * np.log(lmax) / (L4 * DT4)
    ferr = np.abs(f[ok] - f_o)
    print("jacobian: %d of %d valid excluded; rel err median %.2e max %.2e; ftle abs err max %.2e"
          % (excluded, int(both.sum()), np.median(rel), rel.max(), ferr.max()))
    assert rel.max() < JAC_MAX_REL
    assert ferr.max() < FTLE_MAX_ABS
    assert np.all(np.isnan(f[v == 0]))


def test_ftle_of_linear_field_closed_form():
    import torch
    A = np.array([[0.5, 0.25, 0.0], [0.0, -0.25, 0.125], [0.0, 0.0, -0.25]])
    c = np.array([8.0, 8.0, 8.0])
    n, h, L, dt = (16, 16, 16), (1.0,) * 3, 8, 0.125
    field = inputs.affine_field(n, (0, 0, 0), h, A, -A @ c)
    x0 = c + np.array([[0.1, 0.2, -0.3], [-0.25, 0.0, 0.5]])
    tape = adjoint.Tape(n, (0, 0, 0), h, 2, L, 3)
    ends, valid, J, f = adjoint.ftle(tape, torch.from_numpy(x0.astype(np.float32)).cuda(),
                                     _fields_dev([field] * L), dt)
    tape.close()
    M = np.linalg.matrix_power(_R(dt * A), L)
    want = np.log(np.linalg.svd(M, compute_uv=False)[0]) / (L * dt)
    assert np.allclose(J.cpu().numpy(), M[None], rtol=1e-5, atol=1e-6)
    assert np.allclose(f.cpu().numpy(), want, rtol=1e-5)


def test_tape_call_order():
    import torch
    tape = adjoint.Tape((4, 4, 4), (0, 0, 0), (1, 1, 1), 3, 2, 1)
    g = torch.zeros((3, 3), device="cuda")
    with pytest.raises(bto.BtoError) as e:
        bto.bto_tape_backward(tape.handle, g, g)
    assert e.value.status == bto.BTO_ERR_STATE
    F = torch.zeros((2, 5, 5, 5, 3), device="cuda")
    s = torch.full((3, 3), 2.0, device="cuda", requires_grad=True)
    ends, _, _ = adjoint.flow_map(s, F, tape, 0.1)
    adjoint.flow_map(s, F, tape, 0.1)                 # a second forward on the same tape
    with pytest.raises(RuntimeError):
        ends.sum().backward()
    tape.close()
