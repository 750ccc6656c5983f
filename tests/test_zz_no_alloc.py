"""pr_lbvh_build_noalloc: the LBVH build for callers that cannot let the library
allocate device memory during a call (their device memory is owned by their
own allocator under a fixed budget, or they run latency-sensitive loops where
an allocation's synchronisation is unacceptable). It must give exactly what
pr_lbvh_build gives, on two calls in a row (the shared fixed scratch keeps the
previous call's contents), and refuse sizes beyond its fixed limit.

Kept in a file of its own that pytest collects last; it passes alone in a
fresh process (the first call performs the per-device set-up) and after the
other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_10357_b300 as pr  # noqa: E402

MAX_BOXES = 262144


def _boxes(n, seed):
    rng = np.random.default_rng(seed)
    lo = rng.uniform(-50, 50, (n, 3)).astype(np.float32)
    b = np.concatenate([lo, lo + rng.uniform(0, 3, (n, 3)).astype(np.float32)], 1)
    return torch.from_numpy(b).cuda()


def _outputs(n):
    return dict(nodes=torch.full((max(n - 1, 1), 16), -7.0, device="cuda"),
                perm=torch.full((n,), -7, dtype=torch.int32, device="cuda"),
                codes=torch.full((n,), -7, dtype=torch.int32, device="cuda"),
                root=torch.full((8,), -7.0, device="cuda"))


def _call(fn, boxes, out):
    n = int(boxes.shape[0])
    stream = torch.cuda.current_stream().cuda_stream or None
    return fn(ctypes.c_void_p(boxes.data_ptr()), n, ctypes.c_void_p(out["nodes"].data_ptr()),
              ctypes.c_void_p(out["perm"].data_ptr()), ctypes.c_void_p(out["codes"].data_ptr()),
              ctypes.c_void_p(out["root"].data_ptr()), stream)


def _same(a, b, n):
    assert torch.equal(a["perm"], b["perm"]) and torch.equal(a["codes"], b["codes"])
    assert torch.equal(a["root"][[0, 1, 2, 4, 5, 6]], b["root"][[0, 1, 2, 4, 5, 6]])
    if n > 1:
        assert torch.equal(a["nodes"][: n - 1, :14], b["nodes"][: n - 1, :14])


@pytest.mark.parametrize("n", [5, 1024, 1025, 100_000, MAX_BOXES])
def test_noalloc_matches_allocating_build_twice(n):
    lib = pr._lib
    boxes = _boxes(n, seed=n)
    ref = _outputs(n)
    assert _call(lib.pr_lbvh_build, boxes, ref) == pr.PR_OK
    torch.cuda.synchronize()
    for call in range(2):
        got = _outputs(n)
        assert _call(lib.pr_lbvh_build_noalloc, boxes, got) == pr.PR_OK, lib.pr_last_error()
        torch.cuda.synchronize()
        _same(ref, got, n)


def test_noalloc_after_a_different_input_keeps_no_stale_state():
    lib = pr._lib
    a, b = _boxes(60_000, seed=1), _boxes(3_000, seed=2)
    ref = _outputs(3_000)
    assert _call(lib.pr_lbvh_build, b, ref) == pr.PR_OK
    big = _outputs(60_000)
    assert _call(lib.pr_lbvh_build_noalloc, a, big) == pr.PR_OK
    got = _outputs(3_000)
    assert _call(lib.pr_lbvh_build_noalloc, b, got) == pr.PR_OK
    torch.cuda.synchronize()
    _same(ref, got, 3_000)


def test_noalloc_rejects_sizes_beyond_its_limit():
    lib = pr._lib
    n = MAX_BOXES + 1
    boxes = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
    out = _outputs(4)
    assert _call(lib.pr_lbvh_build_noalloc, boxes, out) == pr.PR_ERR_INVALID_ARG
    assert b"exceeds the fixed scratch limit" in lib.pr_last_error()
    torch.cuda.synchronize()
    assert float(out["root"][0]) == -7.0          # nothing was written


def test_noalloc_allocates_nothing():
    """The point of the entry point: once a device has seen its first call,
    calls take no device memory. Around two calls of 100 000 boxes the default
    memory pool's high-water marks stay at zero and the device's free memory
    is unchanged, while one pr_lbvh_build of the same boxes (which takes its
    scratch from that pool) does raise the mark, so the check can see an
    allocation."""
    from cuda.bindings import driver, runtime as cudart
    lib = pr._lib
    err, pool = cudart.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())
    assert err == cudart.cudaError_t.cudaSuccess
    used_high = cudart.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh
    reserved_high = cudart.cudaMemPoolAttr.cudaMemPoolAttrReservedMemHigh

    def reset_marks():
        for attr in (used_high, reserved_high):
            assert cudart.cudaMemPoolSetAttribute(pool, attr, driver.cuuint64_t(0))[0] == cudart.cudaError_t.cudaSuccess

    def mark(attr):
        err, v = cudart.cudaMemPoolGetAttribute(pool, attr)
        assert err == cudart.cudaError_t.cudaSuccess
        return int(v)

    n = 100_000
    boxes = _boxes(n, seed=9)
    outs = [_outputs(n) for _ in range(3)]
    assert _call(lib.pr_lbvh_build_noalloc, boxes, outs[0]) == pr.PR_OK      # first call on the device: set-up
    torch.cuda.synchronize()
    reset_marks()       # the marks restart from the pool's current use (memory earlier tests left in it)
    used0, reserved0 = mark(used_high), mark(reserved_high)
    free_before = torch.cuda.mem_get_info()[0]
    for k in (1, 2):
        assert _call(lib.pr_lbvh_build_noalloc, boxes, outs[k]) == pr.PR_OK
    torch.cuda.synchronize()
    assert mark(used_high) == used0 and mark(reserved_high) == reserved0
    assert torch.cuda.mem_get_info()[0] >= free_before          # the pool may only have given memory back
    _same(outs[0], outs[2], n)
    ref = _outputs(n)
    assert _call(lib.pr_lbvh_build, boxes, ref) == pr.PR_OK                   # the allocating build
    torch.cuda.synchronize()
    assert mark(used_high) > used0
    _same(ref, outs[1], n)
