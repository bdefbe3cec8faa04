"""The allocation-free entry point against the regular one.

rrs_depth_noalloc exists for callers that cannot allocate device memory (plug-ins
inside another framework's pool, processes that forbid allocation once running):
it draws its working memory from a fixed device array inside the library.  It
runs the same kernels as rrs_depth, so on the same inputs its results must equal
rrs_depth's: halfspace counts and depths bit for bit, projection depths within
the 1e-5 relative tolerance used by the other parity tests.  Two calls in a row
check that the contents the shared array keeps from the previous call do not
leak into the next one.  This file is collected last.
"""
import numpy as np
import pytest
import torch

import paper_2506_08262_gb300 as rrs
import workloads

pytestmark = pytest.mark.gpu


def regular(X, Z, kind, k, r, alpha, seed):
    with rrs.Context(0) as ctx:
        did = ctx.register(X)
        dep, cnt, _ = ctx.depth(did, Z, kind, k, r, alpha, seed)
        out = dep.cpu().numpy(), cnt.cpu().numpy()
        ctx.free(did)
    return out


def noalloc(X, Z, kind, k, r, alpha, seed):
    dep = torch.full((Z.shape[0],), -7.0, dtype=torch.float64, device="cuda")
    cnt = torch.full((Z.shape[0],), -7, dtype=torch.int64, device="cuda")
    dt = rrs.RRS_F32 if X.dtype == torch.float32 else rrs.RRS_F64
    rrs.rrs_depth_noalloc(X, X.shape[0], X.shape[1], dt, Z, Z.shape[0], kind, k, r, alpha, seed, dep, cnt,
                          torch.cuda.current_stream())
    return dep.cpu().numpy(), cnt.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def built():
    from __graft_entry__ import build
    build()


@pytest.mark.parametrize("kind", [rrs.RRS_HALFSPACE, rrs.RRS_PROJECTION, rrs.RRS_ASYM_PROJECTION])
def test_noalloc_matches_rrs_depth_two_calls_in_a_row(kind):
    X, Z = workloads.gaussian_cloud(40 + kind, 1537, 7, 23, dtype=np.float32)
    Xd, Zd = torch.from_numpy(X).cuda(), torch.from_numpy(Z).cuda()
    ref_d, ref_c = regular(Xd, Zd, kind, 150, 5, 0.6, 9)
    # a different call first (another cloud, more queries, another seed and direction count), so the
    # scratch holds unrelated contents when the compared calls run; then two compared calls in a row
    X2, Z2 = workloads.gaussian_cloud(70 + kind, 2100, 7, 61, dtype=np.float32)
    noalloc(torch.from_numpy(X2).cuda(), torch.from_numpy(Z2).cuda(), kind, 240, 6, 0.8, 4)
    for _ in range(2):
        got_d, got_c = noalloc(Xd, Zd, kind, 150, 5, 0.6, 9)
        if kind == rrs.RRS_HALFSPACE:
            np.testing.assert_array_equal(got_c, ref_c)
            np.testing.assert_array_equal(got_d, ref_d)
        else:
            np.testing.assert_allclose(got_d, ref_d, rtol=1e-5, atol=0)
            assert np.all(got_c == -1)


def test_noalloc_binding_refuses_bad_buffers():
    # the C entry point takes raw device addresses; the binding refuses what would make the kernels
    # read or write outside a buffer or through a host address
    X = torch.zeros((50, 4), dtype=torch.float32, device="cuda")
    Z = torch.zeros((3, 4), dtype=torch.float32, device="cuda")
    ok_out = torch.zeros(3, dtype=torch.float64, device="cuda")
    cases = [
        dict(X=X.cpu()),                                                  # host tensor
        dict(Z=Z.double()),                                               # dtype differs from X's
        dict(out=torch.zeros(3, dtype=torch.float32, device="cuda")),     # depth_out not float64
        dict(out=torch.zeros(2, dtype=torch.float64, device="cuda")),     # depth_out too short
        dict(cnt=torch.zeros(3, dtype=torch.int32, device="cuda")),       # count_out not int64
        dict(X=torch.zeros((4, 50), dtype=torch.float32, device="cuda").t()),   # not contiguous
        dict(X=np.zeros((50, 4), np.float32)),                            # numpy array
    ]
    for c in cases:
        with pytest.raises(rrs.RRSError) as e:
            rrs.rrs_depth_noalloc(c.get("X", X), 50, 4, rrs.RRS_F32, c.get("Z", Z), 3, rrs.RRS_PROJECTION, 20, 2,
                                  0.5, 0, c.get("out", ok_out), c.get("cnt"))
        assert e.value.status == rrs.RRS_ERR_INVALID_ARG


@pytest.mark.parametrize("kind", [rrs.RRS_PROJECTION, rrs.RRS_ASYM_PROJECTION])
@pytest.mark.parametrize("d", [6, 20])
def test_noalloc_keys_beyond_shared_memory(kind, d):
    # n = 58,000: keys outside shared memory; the allocation-free entry point recomputes them at every
    # pass, the regular one forms them once (keys kernels, same arithmetic) and reads them at every pass
    X, Z = workloads.gaussian_cloud(60 + kind, 58_000, d, 5, dtype=np.float32)
    Xd, Zd = torch.from_numpy(X).cuda(), torch.from_numpy(Z).cuda()
    ref_d, _ = regular(Xd, Zd, kind, 40, 2, 0.7, 3)
    got_d, _ = noalloc(Xd, Zd, kind, 40, 2, 0.7, 3)
    np.testing.assert_allclose(got_d, ref_d, rtol=1e-5, atol=0)


def test_noalloc_fp64_halfspace_and_a_different_second_call():
    # FP64 data (the exact recheck reads the caller's array), then a smaller call after a larger one
    P = workloads.c1()
    Xd, Zd = torch.from_numpy(P.X).cuda(), torch.from_numpy(P.Z).cuda()
    ref_d, ref_c = regular(Xd, Zd, rrs.RRS_HALFSPACE, P.k, P.r, P.alpha, P.seed)
    got_d, got_c = noalloc(Xd, Zd, rrs.RRS_HALFSPACE, P.k, P.r, P.alpha, P.seed)
    np.testing.assert_array_equal(got_c, ref_c)
    np.testing.assert_array_equal(got_d, ref_d)
    small_d, small_c = noalloc(Xd[:100], Zd[:5], rrs.RRS_HALFSPACE, 60, 3, 0.5, 1)
    ref_sd, ref_sc = regular(Xd[:100], Zd[:5], rrs.RRS_HALFSPACE, 60, 3, 0.5, 1)
    np.testing.assert_array_equal(small_c, ref_sc)
    np.testing.assert_array_equal(small_d, ref_sd)


def test_noalloc_rejects_requests_beyond_its_scratch():
    X = torch.zeros((3_000_000, 8), dtype=torch.float32, device="cuda")   # 96 MB > 32 MiB of scratch
    Z = torch.zeros((1, 8), dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(rrs.RRSError) as e:
        rrs.rrs_depth_noalloc(X, X.shape[0], 8, rrs.RRS_F32, Z, 1, rrs.RRS_HALFSPACE, 10, 2, 0.5, 0, out)
    assert e.value.status == rrs.RRS_ERR_BUDGET
    assert "scratch" in str(e.value)
