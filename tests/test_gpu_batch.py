"""GPU parity for the batched grouped launch (ddg_batch_*, dd_gemm_batched).

* Every product of a mixed DD/QD batch of uneven shapes (Block, Strassen and
  Winograd with small cutoffs, all modes, odd sizes) is bit-identical to the
  same product alone through dd_gemm (same kernels, same operation order).
* Graph replays give the same bits as the first run.
* The batch of the batched workload (1000 problems, dims log-uniform in
  [32, 1024], 70% DD / 30% QD) stays within the algorithms' bounds on
  sampled entries against the oracle's exact checker.
"""
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


def make_batch(count, lo, hi, seed, qd_frac=0.3, cutoffs=(8, 16, 40)):
    dims = I.log_uniform_dims(count, lo, hi, seed)
    u = I.uniform01(seed + 1, 4 * count).reshape(count, 4)
    probs = []
    for t in range(count):
        m, l, n = (int(x) for x in dims[t])
        limbs = 4 if u[t, 0] < qd_frac else 2
        algo = ["block", "strassen", "winograd"][int(u[t, 1] * 3)]
        cutoff = cutoffs[int(u[t, 2] * len(cutoffs))]
        mode = ["set", "add", "sub"][int(u[t, 3] * 3)]
        A = I.uniform(m, l, limbs, seed=1000 * seed + 3 * t)
        B = I.uniform(l, n, limbs, seed=1000 * seed + 3 * t + 1)
        C0 = I.uniform(m, n, limbs, seed=1000 * seed + 3 * t + 2)
        probs.append(dict(A=A, B=B, C0=C0, algo=algo, cutoff=cutoff, mode=mode, limbs=limbs))
    return probs


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_bit_identical_to_single_calls(use_graph):
    import paper_1510_08642_gb300 as P
    probs = make_batch(60, 1, 160, seed=7)
    dev = []
    for p in probs:
        dA, dB = to_dev(p["A"]), to_dev(p["B"])
        dev.append((dA, dB, to_dev(p["C0"]), to_dev(p["C0"])))
    plist = [P.problem(dA, dB, dC, p["algo"], p["cutoff"], p["mode"]) for (dA, dB, dC, _), p in zip(dev, probs)]
    batch = P.Batch(plist, use_graph=use_graph)
    assert batch.stats["problems"] == 60
    batch.run()
    for (dA, dB, _, dC1), p in zip(dev, probs):
        P.gemm(dA, dB, dC1, algo=p["algo"], cutoff=p["cutoff"], mode=p["mode"])
    torch.cuda.synchronize()
    for (dA, dB, dC, dC1), p in zip(dev, probs):
        assert np.array_equal(to_host(dC), to_host(dC1)), (p["algo"], p["cutoff"], p["mode"], p["A"].shape)
    if use_graph:  # replays: reset C, run the graph twice more
        first = [to_host(d[2]).copy() for d in dev]
        for _ in range(2):
            for (dA, dB, dC, _), p in zip(dev, probs):
                dC.copy_(to_dev(p["C0"]))
            batch.run()
        torch.cuda.synchronize()
        for d, f in zip(dev, first):
            assert np.array_equal(to_host(d[2]), f)
    batch.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_converted_leaves_bit_identical(use_graph):
    """Larger problems, whose leaves convert their operands once in one
    grouped conversion launch before a grouped product on converted
    operands: the same bits as each product alone, and the conversion
    launch is there (launch profile)."""
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    probs = make_batch(14, 64, 420, seed=9, cutoffs=(64, 100, 200))
    dev = []
    for p in probs:
        dA, dB = to_dev(p["A"]), to_dev(p["B"])
        dev.append((dA, dB, to_dev(p["C0"]), to_dev(p["C0"])))
    plist = [P.problem(dA, dB, dC, p["algo"], p["cutoff"], p["mode"]) for (dA, dB, dC, _), p in zip(dev, probs)]
    batch = P.Batch(plist, use_graph=use_graph)
    if not use_graph:
        capi.ddg_profile_begin()
    batch.run()
    if not use_graph:
        prof = capi.ddg_profile_end()
        assert prof["convert"]["launches"] >= 1 and prof["convert"]["ops"] > 0
    for (dA, dB, _, dC1), p in zip(dev, probs):
        P.gemm(dA, dB, dC1, algo=p["algo"], cutoff=p["cutoff"], mode=p["mode"])
    torch.cuda.synchronize()
    for (dA, dB, dC, dC1), p in zip(dev, probs):
        assert np.array_equal(to_host(dC), to_host(dC1)), (p["algo"], p["cutoff"], p["mode"], p["A"].shape)
    batch.close()


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("recursive", [False, True])
def test_one_leaf_launch_plan_bit_identical(use_graph, recursive):
    """DDG_BATCH_ONE_LEAF_LAUNCH: every base-case product, DD and QD, in one
    persistent grouped launch with tiles converted as staged. The same bits
    as the default plan (which converts larger products' operands once) and
    as each product alone; an all-Block batch is a single kernel per run."""
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    probs = make_batch(24, 3, 300, seed=11, qd_frac=0.4, cutoffs=(16, 64, 100))
    if not recursive:
        for p in probs:
            p["algo"] = "block"
    dev = []
    for p in probs:
        dA, dB = to_dev(p["A"]), to_dev(p["B"])
        dev.append((dA, dB, to_dev(p["C0"]), to_dev(p["C0"])))
    one = P.Batch([P.problem(dA, dB, dC, p["algo"], p["cutoff"], p["mode"])
                   for (dA, dB, dC, _), p in zip(dev, probs)], use_graph=use_graph, one_launch=True)
    ref = P.Batch([P.problem(dA, dB, dC1, p["algo"], p["cutoff"], p["mode"])
                   for (dA, dB, _, dC1), p in zip(dev, probs)], use_graph=use_graph)
    if not recursive:
        assert one.stats["launches_per_run"] == 1
    assert one.stats["leaf_tasks"] == ref.stats["leaf_tasks"]
    if not use_graph:
        capi.ddg_profile_begin()
    one.run()
    if not use_graph:
        prof = capi.ddg_profile_end()
        assert prof["convert"]["launches"] == 0 and prof["block"]["launches"] >= 1
    ref.run()
    torch.cuda.synchronize()
    for (dA, dB, dC, dC1), p in zip(dev, probs):
        assert np.array_equal(to_host(dC), to_host(dC1)), (p["algo"], p["cutoff"], p["mode"], p["A"].shape)
        err = O.gemm_error(p["A"], p["B"], to_host(dC), C0=p["C0"], mode=p["mode"])
        assert O.normwise(err, p["A"], p["B"]) <= normwise_bound(p["A"].shape[2], p["limbs"], p["algo"])
    one.close()
    ref.close()


def test_batch_rejects_unknown_flags():
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    A = to_dev(I.uniform(4, 4, 2, seed=1))
    p = P.problem(A, A, to_dev(I.uniform(4, 4, 2, seed=2)), "block", 8)
    with pytest.raises(capi.DDGError) as e:
        capi.ddg_batch_create([p], False, torch.cuda.current_stream().cuda_stream, flags=2)
    assert e.value.status == capi.DDG_EINVAL


def test_dd_gemm_batched_one_shot():
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    probs = make_batch(12, 5, 90, seed=8, qd_frac=0.5)
    dev, plist, keep = [], [], []
    for p in probs:
        dA, dB, dC = to_dev(p["A"]), to_dev(p["B"]), to_dev(p["C0"])
        keep += [dA, dB]  # the problems hold raw pointers: keep the operands alive
        dev.append(dC)
        plist.append(P.problem(dA, dB, dC, p["algo"], p["cutoff"], p["mode"]))
    capi.check(capi.dd_gemm_batched(plist, torch.cuda.current_stream().cuda_stream))
    for dC, p in zip(dev, probs):
        err = O.gemm_error(p["A"], p["B"], to_host(dC), C0=p["C0"], mode=p["mode"])
        assert O.normwise(err, p["A"], p["B"]) <= normwise_bound(p["A"].shape[2], p["limbs"], p["algo"])


def test_batch_rejects_bad_problem():
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    A = to_dev(I.uniform(4, 4, 2, seed=1))
    p = P.problem(A, A, to_dev(I.uniform(4, 4, 2, seed=2)), "simple", 8)
    with pytest.raises(capi.DDGError) as e:
        P.Batch([p])
    assert e.value.status == capi.DDG_EINVAL


def test_batched_workload_1000_problems():
    """1000 products, dims log-uniform in [32, 1024], 70% DD / 30% QD."""
    import paper_1510_08642_gb300 as P
    count = 1000
    dims = I.log_uniform_dims(count, 32, 1024, seed=4)
    kind = I.uniform01(5, count)
    dev, plist, host = [], [], []
    for t in range(count):
        m, l, n = (int(x) for x in dims[t])
        limbs = 4 if kind[t] < 0.3 else 2
        A = I.uniform(m, l, limbs, seed=10 * t + 1)
        B = I.uniform(l, n, limbs, seed=10 * t + 2)
        dA, dB = to_dev(A), to_dev(B)
        dC = torch.empty((limbs, m, n), dtype=torch.float64, device="cuda")
        algo = "winograd" if min(m, l, n) > 256 else "block"
        plist.append(P.problem(dA, dB, dC, algo, 256))
        dev.append((dA, dB, dC))
        host.append((A, B, algo, limbs))
    batch = P.Batch(plist, use_graph=True)
    batch.run()
    batch.run()
    torch.cuda.synchronize()
    for t in range(0, count, 37):  # sampled problems, sampled entries
        A, B, algo, limbs = host[t]
        C = to_host(dev[t][2])
        rows, cols = sample_entries(A.shape[1], B.shape[2], 16, seed=t)
        err = O.gemm_error(A, B, C, rows=rows, cols=cols)
        scale = np.linalg.norm(A[0]) * np.linalg.norm(B[0])
        assert np.all(np.abs(err) <= normwise_bound(A.shape[2], limbs, algo) * scale)
    batch.close()
