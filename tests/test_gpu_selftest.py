"""Numerical building blocks of the kernels, on the GPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_reciprocal_within_one_ulp():
    """The row-tiled kernels form u = j / rho with 1/rho from the hardware's
    approximate reciprocal refined by one Newton-Raphson step. Against the
    correctly rounded FP32 reciprocal (numpy, IEEE division) it must be within one
    ulp over the densities the method meets (rho in [0.25, 4]) and beyond."""
    import __graft_entry__
    __graft_entry__.build()
    import ctypes
    import torch
    from paper_1111_2142_gb300 import lwacm as lw
    lib = lw.load()
    rng = np.random.default_rng(5)
    # every float in [1, 1 + 2^-7) (a dense sweep of mantissas), plus random
    # values log-uniform on [1/64, 64]
    dense = (np.arange(1 << 16, dtype=np.uint32) + np.float32(1.0).view(np.uint32)).view(np.float32)
    rand = np.exp(rng.uniform(np.log(1 / 64), np.log(64), 1 << 20)).astype(np.float32)
    x = np.concatenate([dense, rand, np.float32([0.25, 0.5, 1.0, 2.0, 4.0])])
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    st = torch.cuda.current_stream()
    assert lib.lwacm_selftest_reciprocal(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         x.size, ctypes.c_void_p(st.cuda_stream)) == lw.OK
    got = out.cpu().numpy()
    ref = np.float32(1.0) / x
    ulps = np.abs(got.view(np.int32).astype(np.int64) - ref.view(np.int32).astype(np.int64))
    exact = float(np.mean(ulps == 0))
    print(f"reciprocal: {x.size} values, max {int(ulps.max())} ulp, {100 * exact:.2f}% correctly rounded")
    assert ulps.max() <= 1
    assert np.array_equal(got[-5:], ref[-5:])  # powers of two are exact
