"""Differentiable typed pack: forward = float32 pack, backward = the adjoint
of the pack (scatter-add).  Checked against the oracle's FP64 adjoint
(bit-exact when no entry repeats, within 1e-6 relative when entries repeat),
against exact finite differences, and with torch.autograd.gradcheck."""
import numpy as np
import pytest

import oracle
import inputs

torch = pytest.importorskip("torch")
import paper_2402_12274_gb300 as dte  # noqa: E402
from paper_2402_12274_gb300.autograd import typed_pack  # noqa: E402

pytestmark = pytest.mark.gpu


def six_faces(n, g, rng, repeat_frac):
    specs = inputs.halo_indexed_specs(rng, n=n, g=g, repeat_frac=repeat_frac)
    return inputs.all_faces_struct(specs)


def run_pack_and_adjoint(spec, n_field, rng, count=1):
    t = dte.Datatype.from_spec(spec).commit()
    o = oracle.from_spec(spec)
    x_np = rng.standard_normal(n_field).astype(np.float32)
    x = torch.from_numpy(x_np).cuda().requires_grad_(True)
    y = typed_pack(x, t, count)
    ref = o.pack(x_np.view(np.uint8), count).view(np.float32)
    assert np.array_equal(y.detach().cpu().numpy(), ref)
    gy_np = rng.standard_normal(y.numel()).astype(np.float32)
    y.backward(torch.from_numpy(gy_np).cuda())
    gx = x.grad.cpu().numpy().astype(np.float64)
    want = o.pack_adjoint_f64(gy_np.astype(np.float64), count, n_field)
    return gx, want, o


def test_adjoint_bit_exact_without_repeats():
    rng = np.random.default_rng(501)
    n = 24
    # one face (entries distinct), a vector layout and a strided subarray
    specs = [inputs.halo_indexed_specs(rng, n=n, g=2, repeat_frac=0.0)[k] for k in (0, 3, 5)]
    specs += [("vector", 50, 3, 7, ("basic", "float32")),
              ("subarray", np.array([n, n, n]), np.array([n, 2, n]), np.array([0, 5, 0]), 0, ("basic", "float32"))]
    for spec in specs:
        gx, want, o = run_pack_and_adjoint(spec, n ** 3, rng)
        assert not o.overlaps(1)
        assert np.array_equal(gx, want)


def test_adjoint_repeated_entries_within_1e6():
    rng = np.random.default_rng(502)
    n = 32
    spec = six_faces(n, 2, rng, 0.10)
    gx, want, o = run_pack_and_adjoint(spec, n ** 3, rng)
    assert o.overlaps(1)
    scale = np.maximum(np.abs(want), 1e-30)
    assert np.all(np.abs(gx - want) <= 1e-6 * scale)
    # cells with one source are exact
    single = np.isclose(want, 0) | (np.abs(gx - want) == 0)
    assert single.mean() > 0.5


def test_adjoint_matches_finite_differences():
    rng = np.random.default_rng(503)
    n = 16
    spec = six_faces(n, 2, rng, 0.10)
    t = dte.Datatype.from_spec(spec).commit()
    # small-integer field: x +- 1 is exact in float32, so central differences
    # of the linear map f(x) = <pack(x), y> are exact in FP64
    x_np = rng.integers(-8, 9, n ** 3).astype(np.float32)
    y32 = rng.standard_normal(t.size // 4).astype(np.float32)  # gradient seed

    def f(xv):
        xt = torch.from_numpy(xv).cuda()
        return float(np.dot(typed_pack(xt, t).cpu().numpy().astype(np.float64), y32.astype(np.float64)))

    x = torch.from_numpy(x_np).cuda().requires_grad_(True)
    typed_pack(x, t).backward(torch.from_numpy(y32).cuda())
    gx = x.grad.cpu().numpy().astype(np.float64)
    touched = np.flatnonzero(gx)
    picks = np.concatenate([rng.choice(touched, 48, replace=False), rng.choice(n ** 3, 16, replace=False)])
    for i in picks:
        xp, xm = x_np.copy(), x_np.copy()
        xp[i] += 1
        xm[i] -= 1
        fd = (f(xp) - f(xm)) / 2.0
        assert abs(gx[i] - fd) <= 1e-6 * max(abs(fd), 1e-12), (i, gx[i], fd)


def test_gradcheck_small_field():
    rng = np.random.default_rng(504)
    n = 8
    spec = six_faces(n, 2, rng, 0.10)
    t = dte.Datatype.from_spec(spec).commit()
    x = torch.from_numpy(rng.standard_normal(n ** 3).astype(np.float32)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v: typed_pack(v, t), (x,), eps=1e-2, atol=1e-3, rtol=1e-3,
                                    nondet_tol=0.0)


def test_full_size_halo_with_repeats():
    # 256^3 float32 field, six element-granular faces with 10% repeated entries
    rng = np.random.default_rng(5)
    n = 256
    spec = six_faces(n, 2, rng, 0.10)
    gx, want, o = run_pack_and_adjoint(spec, n ** 3, rng)
    scale = np.maximum(np.abs(want), 1e-30)
    assert np.all(np.abs(gx - want) <= 1e-6 * scale)


def test_adjoint_argument_errors():
    t = dte.Datatype.vector(4, 3, 5, dte.INT16).commit()  # 6-byte runs: not whole floats
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(dte.DteError) as e:
        dte.dte_pack_adjoint_f32_enqueue(buf.data_ptr(), 1, t.h, buf.data_ptr())
    assert e.value.code == dte.ERR_ARG
