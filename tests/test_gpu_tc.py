"""tcgen05 tensor-core GEMM against FP64 numpy on BF16-rounded inputs (GPU required)."""

import ctypes as C

import numpy as np
import pytest
import torch

import paper_2503_22588_gb300 as nbt
from paper_2503_22588_gb300 import _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nbt.build()


def tc_error():
    f = C.c_int32()
    assert _lib.lib().nbt_tc_error(C.byref(f)) == 0
    return f.value


@pytest.mark.parametrize("m,n,k", [(128, 16, 64), (200, 48, 104), (1000, 256, 640), (257, 128, 1728),
                                   (64, 32, 16), (3000, 64, 864), (130, 200, 8), (128, 256, 4160)])
def test_gemm_matches_fp64(m, n, k):
    g = torch.Generator().manual_seed(m * 7 + n * 3 + k)
    a = torch.randn(m, k, generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, generator=g).to(torch.bfloat16)
    ref = a.double().numpy() @ b.double().numpy().T
    ad, bd = a.cuda(), b.cuda()
    c = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    assert _lib.lib().nbt_tc_gemm(ad.data_ptr(), bd.data_ptr(), c.data_ptr(), m, n, k,
                                   torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert tc_error() == 0
    got = c.cpu().double().numpy()
    scale = np.sqrt(k) * 1.0
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref)) <= 1e-5 * scale * 4, np.max(np.abs(got - ref))
