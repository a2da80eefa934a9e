"""The tensor-core building block alone (include/donof_testing.h): with integer-valued fp16
operands (and a low part of multiples of 1/64) every product and partial sum is exact in
fp32, so the result must equal the double-precision product exactly, for A given K-major
(128-byte swizzle), MN-major, and K-major interleaved by 8 (no swizzle, core matrices),
ragged K (zero fill past the end) and one or several M tiles, on single CTAs and on CTA pairs
(cta_group::2, 256-row tiles).  Also the bounded device
wait: run out on purpose, it reports DONOF_ERR_TIMEOUT, ends the other role's wait through
the abort flag, and leaves the context usable."""
import ctypes
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_06142_gb300.build as b
    b.build()
    import paper_2004_06142_gb300.binding as bd
    L = bd.lib()
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    L.donof_testing_tc_gemm.argtypes = [vp] * 5 + [i32] * 3 + [vp]
    L.donof_testing_tc_gemm_mn.argtypes = [vp] * 5 + [i32] * 3 + [vp]
    L.donof_testing_tc_gemm_il8.argtypes = [vp] * 5 + [i32] * 3 + [vp]
    L.donof_testing_tc_gemm_ex.argtypes = [vp] * 5 + [i32] * 5 + [vp]
    L.donof_testing_status.argtypes = [vp]
    L.donof_testing_wait_timeout.argtypes = [ctypes.c_int64, ctypes.c_int64, vp]
    return L


def _half_dev(a):
    import torch
    bits = np.ascontiguousarray(a.astype(np.float16)).view(np.int16)
    return torch.from_numpy(bits.copy()).cuda()


@pytest.mark.parametrize("M,N,K", [(128, 160, 128), (256, 160, 200), (64, 32, 64),
                                   (192, 48, 72)])
@pytest.mark.parametrize("layout", ["k_major", "mn_major", "il8"])
def test_split_product_exact(lib, M, N, K, layout):
    import torch
    rng = np.random.default_rng(M + N + K)
    Ah = rng.integers(-8, 9, (M, K)).astype(np.float64)
    Al = rng.integers(-8, 9, (M, K)) / 64.0
    Bh = rng.integers(-8, 9, (N, K)).astype(np.float64)
    Bl = rng.integers(-8, 9, (N, K)) / 64.0
    ref = Ah @ Bh.T + Ah @ Bl.T + Al @ Bh.T
    if layout == "mn_major":
        a_h, a_l = Ah.T, Al.T
    elif layout == "il8":  # [K/8][M][8]
        a_h, a_l = (x.reshape(M, K // 8, 8).transpose(1, 0, 2) for x in (Ah, Al))
    else:
        a_h, a_l = Ah, Al
    dah, dal, dbh, dbl = _half_dev(a_h), _half_dev(a_l), _half_dev(Bh), _half_dev(Bl)
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    fn = {"k_major": lib.donof_testing_tc_gemm, "mn_major": lib.donof_testing_tc_gemm_mn,
          "il8": lib.donof_testing_tc_gemm_il8}[layout]
    rc = fn(dah.data_ptr(), dal.data_ptr(), dbh.data_ptr(), dbl.data_ptr(), D.data_ptr(), M, N,
            K, s)
    assert rc == 0
    assert lib.donof_testing_status(s) == 0
    np.testing.assert_array_equal(D.cpu().numpy().astype(np.float64), ref)


@pytest.mark.parametrize("M,N,K", [(256, 160, 200), (384, 160, 128), (128, 48, 72),
                                   (512, 144, 1216)])
@pytest.mark.parametrize("layout", [0, 1, 2])
def test_pair_product_exact(lib, M, N, K, layout):
    # the cta_group::2 path (a CTA pair per 256-row tile, each CTA staging half of B): the same
    # exact products, with an odd number of 128-row tiles (the second CTA of the last pair
    # has no rows) and a long K
    import torch
    rng = np.random.default_rng(7 * M + N + K)
    Ah = rng.integers(-8, 9, (M, K)).astype(np.float64)
    Al = rng.integers(-8, 9, (M, K)) / 64.0
    Bh = rng.integers(-8, 9, (N, K)).astype(np.float64)
    Bl = rng.integers(-8, 9, (N, K)) / 64.0
    ref = Ah @ Bh.T + Ah @ Bl.T + Al @ Bh.T
    if layout == 1:
        a_h, a_l = Ah.T, Al.T
    elif layout == 2:
        a_h, a_l = (x.reshape(M, K // 8, 8).transpose(1, 0, 2) for x in (Ah, Al))
    else:
        a_h, a_l = Ah, Al
    dah, dal, dbh, dbl = _half_dev(a_h), _half_dev(a_l), _half_dev(Bh), _half_dev(Bl)
    s = torch.cuda.current_stream().cuda_stream
    for pair in (1, 0):
        D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        rc = lib.donof_testing_tc_gemm_ex(dah.data_ptr(), dal.data_ptr(), dbh.data_ptr(),
                                          dbl.data_ptr(), D.data_ptr(), M, N, K, layout, pair, s)
        assert rc == 0
        assert lib.donof_testing_status(s) == 0
        np.testing.assert_array_equal(D.cpu().numpy().astype(np.float64), ref)


def test_bounded_wait_runs_out_and_context_survives(lib):
    import torch
    import paper_2004_06142_gb300.binding as bd
    s = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    t0 = time.time()
    assert lib.donof_testing_wait_timeout(20_000_000, 5_000_000_000, s) == 0  # 20 ms, 5 s
    st = lib.donof_testing_status(s)
    dt = time.time() - t0
    assert st == -6, bd.donof_status_string(st)  # DONOF_ERR_TIMEOUT
    assert dt < 1.0, dt  # the 5 s wait ended on the abort flag
    assert lib.donof_testing_status(s) == 0  # the status word was cleared
    test_split_product_exact(lib, 128, 160, 128, "k_major")  # the context still works
