"""Uneven batches and the n = 48 / 96 grids (FFT length 96 / 192, radix-3 stages).

The oracle pads to the next power of two (L = 128 / 256) while the library uses
L = 2n, so agreement also checks that the result does not depend on L.
"""
import numpy as np
import pytest

import oracle
import spm_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def spm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_02297_gb300 as spm
    return spm


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("n", [48, 96])
def test_radix3_grids_match_oracle(spm, n):
    k = si.wavenumber_for_grid(n)
    eps, grad = si.medium_bumps(n, seed=n, count=8)
    P = spm.Problem(n, k, eps, grad)
    m, p = oracle.medium(eps, grad)
    x = si.random_field(n, 5)
    ref = oracle.apply_fft(n, k, m, p, x)
    y = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    P.apply_A(torch.from_numpy(x).to("cuda"), y)
    y64 = torch.zeros(x.shape, dtype=torch.complex64, device="cuda")
    P.apply_A(torch.from_numpy(x).to("cuda").to(torch.complex64), y64)
    torch.cuda.synchronize()
    e128 = rel(y.cpu().numpy(), ref)
    e64 = rel(y64.cpu().numpy().astype(np.complex128) - x, ref - x)
    print(f"n={n}: c128 {e128:.2e}, c64 (A-I)x {e64:.2e}")
    assert e128 < 1e-12
    assert e64 < 2e-5


def test_uneven_batch_apply_and_graph_replay(spm):
    probs = [dict(n=n, omega=si.wavenumber_for_grid(n), medium=si.medium_bumps(n, seed=10 + i, count=8))
             for i, n in enumerate([8, 48, 16, 32])]
    B = spm.Batch([q["n"] for q in probs], [q["omega"] for q in probs], [q["medium"][0] for q in probs],
                  [q["medium"][1] for q in probs])
    xs = [torch.from_numpy(si.random_field(q["n"], 40 + i)).to("cuda") for i, q in enumerate(probs)]
    ys = [torch.zeros_like(x) for x in xs]
    refs = []
    for q, x in zip(probs, xs):
        m, p = oracle.medium(*q["medium"])
        refs.append(oracle.apply_fft(q["n"], q["omega"], m, p, x.cpu().numpy()))
    for call in range(3):  # first call runs directly and captures, later calls replay the graph
        for y in ys:
            y.zero_()
        B.apply_A(xs, ys)
        torch.cuda.synchronize()
        for y, r in zip(ys, refs):
            assert rel(y.cpu().numpy(), r) < 1e-12


def test_uneven_batch_solve(spm):
    ns = [16, 48, 32]
    probs = [dict(n=n, omega=si.wavenumber_for_grid(n), medium=si.medium_bumps(n, seed=20 + i, count=8))
             for i, n in enumerate(ns)]
    B = spm.Batch(ns, [q["omega"] for q in probs], [q["medium"][0] for q in probs], [q["medium"][1] for q in probs])
    B.build_stencils(spm.SPM_C64)
    gs, xs = [], []
    for i, q in enumerate(probs):
        e = torch.from_numpy(si.plane_wave(q["n"], q["omega"], (0, 0, 1), (1, 0, 0))).to("cuda")
        g = torch.zeros_like(e)
        B.problems[i].rhs_from_incident(e, g)
        gs.append(g)
        xs.append(torch.zeros_like(g))
    infos, st = B.solve(gs, xs, prec=spm.SPM_MIXED, tol=1e-6)
    for i, q in enumerate(probs):
        assert infos[i].true_relres <= 1e-6
        m, p = oracle.medium(*q["medium"])
        gh = gs[i].cpu().numpy()
        r = gh - oracle.apply_fft(q["n"], q["omega"], m, p, xs[i].cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(gh) <= 1e-6
        print(f"n={q['n']}: iterations {infos[i].iterations}, relres {infos[i].true_relres:.2e}")
