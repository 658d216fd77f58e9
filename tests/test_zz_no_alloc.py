"""eot_marginals_noalloc: the marginals for callers that cannot allocate device
memory. It takes no handle and keeps its scratch space in a fixed array inside
the library, so these tests check, through the C ABI, that it returns what the
allocating entry point eot_marginals returns, on two calls in a row (the second
with other sizes and inputs, over scratch left by the first), within the
tolerances the other GPU tests use. This file is named so that pytest collects
it last; it passes alone in a fresh process as well as after the other tests."""
import numpy as np
import pytest

from oracle import eot_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype)


def _inputs(seed, n, m, gamma, f32):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, size=(n, m))
    if f32:
        C = C.astype(np.float32)
    r = rng.dirichlet(np.ones(n))
    c = rng.dirichlet(np.ones(m))
    u = np.log(r) + rng.normal(0, 0.3, n) + 3.0
    v = np.log(c) - O.lse_c(u[:, None] - gamma * C.astype(np.float64))
    return C, u, v


@pytest.mark.parametrize("prec", ["mixed", "plain_fp32", "fp64"])
def test_noalloc_matches_allocating_entry_point_twice(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_02067_gb300 as E
    from paper_2504_02067_gb300.binding import eot_marginals_noalloc
    E.build()
    f32 = prec != "fp64"
    gamma = 512.0
    tol = 1e-6 if f32 else 1e-12
    h = E.Handle(0, 64, 64)
    try:
        for call, (n, m) in enumerate([(1000, 1024), (300, 517)]):
            C, u, v = _inputs(100 + call, n, m, gamma, f32)
            prob = E.Problem(_t(C, torch.float32 if f32 else torch.float64), precision=prec)
            ud, vd = _t(u), _t(v)
            r_ref, c_ref, _, _, _ = h.marginals(prob, ud, vd, gamma)
            r = torch.full((n,), float("nan"), dtype=torch.float64, device=DEV)
            c = torch.full((m,), float("nan"), dtype=torch.float64, device=DEV)
            status = torch.full((1,), -1, dtype=torch.int32, device=DEV)
            eot_marginals_noalloc(prob, ud, vd, gamma, r, c, status)
            torch.cuda.synchronize()
            assert status.item() == 0
            assert (r - r_ref).abs().sum().item() <= tol
            assert (c - c_ref).abs().sum().item() <= tol
    finally:
        h.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_02067_gb300 as E
    from paper_2504_02067_gb300.binding import EotError, eot_marginals_noalloc
    E.build()
    n = 16385
    C = torch.zeros(n, 4, dtype=torch.float32, device=DEV)
    prob = E.Problem(C, precision="mixed")
    u = torch.zeros(n, dtype=torch.float64, device=DEV)
    v = torch.zeros(4, dtype=torch.float64, device=DEV)
    with pytest.raises(EotError):
        eot_marginals_noalloc(prob, u, v, 1.0, torch.empty_like(u), torch.empty_like(v))


def test_noalloc_at_its_size_limit_with_unaligned_rows():
    """n = m = 16384, the largest size the fixed scratch array serves, with a
    leading dimension m + 1 (16-byte loads impossible: the scalar path with the
    most column strips and tickets), compared with eot_marginals on the same
    seeded inputs; then m = 16385 is rejected."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_02067_gb300 as E
    from paper_2504_02067_gb300.binding import EotError, eot_marginals_noalloc
    E.build()
    n = m = 16384
    gen = torch.Generator(device=DEV).manual_seed(7)
    Cfull = torch.rand(n, m + 1, generator=gen, device=DEV, dtype=torch.float32)
    C = Cfull[:, :m]
    assert C.stride(0) == m + 1
    gamma = 8.0
    u = (torch.randn(n, generator=gen, device=DEV, dtype=torch.float64) * 0.3 - np.log(n))
    v = (torch.randn(m, generator=gen, device=DEV, dtype=torch.float64) * 0.3 - np.log(m))
    prob = E.Problem(C, precision="mixed")
    h = E.Handle(0, 64, 64)
    try:
        r_ref, c_ref, _, _, _ = h.marginals(prob, u, v, gamma)
    finally:
        h.close()
    for call in range(2):
        r = torch.full((n,), float("nan"), dtype=torch.float64, device=DEV)
        c = torch.full((m,), float("nan"), dtype=torch.float64, device=DEV)
        status = torch.full((1,), -1, dtype=torch.int32, device=DEV)
        eot_marginals_noalloc(prob, u, v, gamma, r, c, status)
        torch.cuda.synchronize()
        assert status.item() == 0
        mass = r_ref.sum().item()
        assert (r - r_ref).abs().sum().item() <= 1e-6 * mass
        assert (c - c_ref).abs().sum().item() <= 1e-6 * mass
    del Cfull, C
    Cw = torch.zeros(4, 16385, dtype=torch.float32, device=DEV)
    probw = E.Problem(Cw, precision="mixed")
    uw = torch.zeros(4, dtype=torch.float64, device=DEV)
    vw = torch.zeros(16385, dtype=torch.float64, device=DEV)
    with pytest.raises(EotError):
        eot_marginals_noalloc(probw, uw, vw, 1.0, torch.empty_like(uw), torch.empty_like(vw))
