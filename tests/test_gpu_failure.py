"""Failure detection of the tensor-core kernels (GPU required): a bounded device-side wait runs out.

Every mbarrier wait of the tcgen05 kernels is bounded by a limit on the GPU's global timer.  When
a wait gives up, the kernel sets the library's device error word, waits (bounded) for its own
tensor-core work in flight, frees its tensor memory and returns, so the CUDA context stays usable.
Here the limit is shortened to 1 ms and a probe kernel waits on an mbarrier that nothing completes
(no fault, trap or hang is involved): the launch ends, the error word is set, and ordinary
tensor-core work on the same context afterwards is correct and leaves the word clear.
"""

import ctypes as C
import time

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


def _error_word():
    f = C.c_int32()
    assert _lib.lib().nbt_tc_error(C.byref(f)) == 0
    return f.value


def _gemm_ok():
    g = torch.Generator(device="cuda").manual_seed(0)
    a = torch.randn((200, 64), device="cuda", generator=g).to(torch.bfloat16)
    b = torch.randn((48, 64), device="cuda", generator=g).to(torch.bfloat16)
    c = torch.empty((200, 48), dtype=torch.float32, device="cuda")
    assert _lib.lib().nbt_tc_gemm(a.data_ptr(), b.data_ptr(), c.data_ptr(), 200, 48, 64, None) == 0
    torch.cuda.synchronize()
    want = a.double().cpu().numpy() @ b.double().cpu().numpy().T
    return np.allclose(c.cpu().numpy(), want, rtol=1e-5, atol=1e-4)


def test_a_wait_that_runs_out_sets_the_error_word_and_frees_tensor_memory():
    L = _lib.lib()
    assert _error_word() == 0
    assert L.nbt_tc_set_wait_limit(10) == -1            # below the accepted range
    assert L.nbt_tc_set_wait_limit(10 ** 12) == -1      # above it
    try:
        assert L.nbt_tc_set_wait_limit(1_000_000) == 0  # 1 ms
        t0 = time.perf_counter()
        assert L.nbt_tc_wait_probe(None) == 0
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    finally:
        assert L.nbt_tc_set_wait_limit(2_000_000_000) == 0
    assert dt < 5.0, dt
    assert _error_word() == 1                           # the wait gave up and said so
    assert _error_word() == 0                           # reading cleared it
    # every SM's tensor memory was freed: GEMMs (which allocate it on every SM they run on) complete
    for _ in range(3):
        assert _gemm_ok()
    assert _error_word() == 0


def test_the_probe_twice_in_a_row_and_then_the_surrogate_still_works():
    from oracle import surrogate as S
    from paper_2503_22588_gb300 import surrogate as gs
    L = _lib.lib()
    try:
        assert L.nbt_tc_set_wait_limit(2_000_000) == 0
        assert L.nbt_tc_wait_probe(None) == 0
        assert L.nbt_tc_wait_probe(None) == 0
        torch.cuda.synchronize()
    finally:
        assert L.nbt_tc_set_wait_limit(2_000_000_000) == 0
    assert _error_word() == 1
    crops = torch.zeros((4, 32, 32, 32), dtype=torch.uint8, device="cuda")
    crops[:, :, :16] = 2
    feats = torch.ones((4, 8), dtype=torch.bfloat16, device="cuda")
    net = gs.Surrogate(max_batch=4, params=S.init_params(1))
    y = net.forward(crops, feats)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()
    assert _error_word() == 0
    net.close()
