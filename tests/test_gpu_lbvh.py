"""Standalone device LBVH (pr_lbvh_build) vs the FP32 reference LBVH, bit for bit.

Covers the one-CTA path (n <= 1024) and the radix-sort path (n > 1024), the
boundary sizes, duplicate boxes (equal Morton codes), all-identical boxes
(zero centroid extent: every code is 0) and flat sets (zero extent on an axis).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_10357_b300 as pr  # noqa: E402
import oracle  # noqa: E402


def _boxes(n, kind, seed):
    rng = np.random.default_rng(seed)
    lo = rng.uniform(-50, 50, (n, 3)).astype(np.float32)
    ext = rng.uniform(0, 3, (n, 3)).astype(np.float32)
    if kind == "dup":
        lo[n // 2:] = lo[: n - n // 2]
        ext[n // 2:] = ext[: n - n // 2]
    elif kind == "same":
        lo[:] = lo[0]
        ext[:] = ext[0]
    elif kind == "flat":
        lo[:, 1] = 7.0
        ext[:, 1] = 0.0
    return np.concatenate([lo, lo + ext], 1)


def compare_to_reference(got, ref, label):
    n = len(ref["perm"])
    assert np.array_equal(got["perm"], ref["perm"]), label
    assert np.array_equal(got["codes"], ref["codes"]), label
    if n > 1:
        rc = ref["child"].astype(np.int64)
        mapped = np.where(rc < 0, (0x80000000 | ref["perm"][rc & 0x7FFFFFFF].astype(np.int64)) - (1 << 32), rc)
        assert np.array_equal(got["child"].astype(np.int64), mapped), label
        assert np.array_equal(got["cbox"], ref["cbox"]), label
    assert np.array_equal(got["root"], ref["root"]), label


@pytest.mark.parametrize("n", [1, 2, 3, 17, 1000, 1024, 1025, 2048, 5000, 100_000])
@pytest.mark.parametrize("kind", ["random", "dup"])
def test_lbvh_build_matches_reference(n, kind):
    b = _boxes(n, kind, seed=n)
    res = pr.lbvh_build(torch.from_numpy(b).cuda())
    torch.cuda.synchronize()
    compare_to_reference(pr.lbvh_to_host(res), oracle.lbvh_f32(b), f"{kind} n={n}")


@pytest.mark.parametrize("n", [5, 4000])
@pytest.mark.parametrize("kind", ["same", "flat"])
def test_lbvh_build_degenerate_sets(n, kind):
    b = _boxes(n, kind, seed=7)
    res = pr.lbvh_build(torch.from_numpy(b).cuda())
    torch.cuda.synchronize()
    got = pr.lbvh_to_host(res)
    compare_to_reference(got, oracle.lbvh_f32(b), f"{kind} n={n}")
    if kind == "same":
        assert (got["codes"] == 0).all()


def test_lbvh_build_empty_is_a_no_op():
    res = pr.lbvh_build(torch.zeros((0, 6), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert res["perm"].numel() == 0


def test_lbvh_build_repeated_calls_are_identical():
    b = torch.from_numpy(_boxes(30000, "random", seed=3)).cuda()
    first = pr.lbvh_to_host(pr.lbvh_build(b))
    for _ in range(3):
        again = pr.lbvh_to_host(pr.lbvh_build(b))
        for k in first:
            assert np.array_equal(first[k], again[k])
