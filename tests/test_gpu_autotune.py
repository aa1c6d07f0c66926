"""The autotuner on the GPU: tune() on two shape buckets stores a choice
that choose() then returns for other shapes of those buckets (and after a
save / load), and the chosen configurations' results stay within their
bounds against the exact checker; tune_product() with normwise accuracy
allowed picks among the elementwise algorithms and the tensor-core CRT
product with the fewest moduli that meet the requested precision."""
import numpy as np
import pytest

import oracle as O
from paper_1510_08642_gb300 import inputs as I
from tests.gpu_util import normwise_bound, sample_entries, to_dev, to_host

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_tune_two_buckets_then_choose_and_bounds(tmp_path):
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import autotune
    path = str(tmp_path / "tune.json")
    t = autotune.Tuner(path)
    chosen = {}
    for limbs, (m, l, n) in [(2, (300, 280, 260)), (4, (140, 130, 120))]:
        algo, cutoff = t.tune(limbs, m, l, n, copies=2, reps=2)
        chosen[limbs] = (algo, cutoff)
        assert (algo, cutoff) in t.candidates(m, l, n)
        # another shape of the same bucket gets the stored choice
        assert t.choose(limbs, m + 7, l - 5, n + 3) == (algo, cutoff)
    t.save()
    t2 = autotune.Tuner(path)
    for limbs, (m, l, n) in [(2, (300, 280, 260)), (4, (140, 130, 120))]:
        assert t2.choose(limbs, m, l, n) == chosen[limbs]
        A = I.uniform(m, l, limbs, seed=300 + limbs)
        B = I.uniform(l, n, limbs, seed=310 + limbs)
        C = torch.zeros((limbs, m, n), dtype=torch.float64, device="cuda")
        algo, cutoff = t2.choose(limbs, m, l, n)
        b = P.Batch([P.problem(to_dev(A), to_dev(B), C, algo, cutoff)])
        b.run()
        torch.cuda.synchronize()
        err = O.gemm_error(A, B, to_host(C))
        assert O.normwise(err, A, B) <= normwise_bound(l, limbs, algo)
        b.close()


def test_tune_product_normwise_choice_within_bound(tmp_path):
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import autotune, capi
    t = autotune.Tuner(str(tmp_path / "tune.json"))
    m = l = n = 1024
    cands = t.product_candidates(2, m, l, n, allow_normwise=True, bits=104)
    tc = [c for c in cands if c["algo"] == "ozaki2_tc"]
    assert len(tc) == 1 and tc[0]["slices"] == autotune.moduli_for(l, 104)
    choice = t.tune_product(2, m, l, n, allow_normwise=True, bits=104, reps=2)
    assert t.choose_product(2, m, l, n, allow_normwise=True) == choice
    A = I.uniform(m, l, 2, seed=320)
    B = I.uniform(l, n, 2, seed=321)
    C = to_host(P.gemm(to_dev(A), to_dev(B), **choice))
    rows, cols = sample_entries(m, n, 24, seed=5)
    err = O.gemm_error(A, B, C, rows=rows, cols=cols)
    if choice["algo"] == "ozaki2_tc":
        Pbits = capi.ddg_ozaki2_precision(choice["slices"], l)
        assert Pbits >= 104 + 10
        assert np.all(np.abs(err) <= l * 2.0 ** -Pbits + 2.0 ** -104 * np.abs(C[0][rows, cols]))
    else:
        scale = np.linalg.norm(A[0]) * np.linalg.norm(B[0])
        assert np.all(np.abs(err) <= normwise_bound(l, 2, choice["algo"]) * scale)
