"""mickey_init_state_noalloc against the regular key/IV loading.

The allocation-free entry point serves callers that may not allocate device
memory (an application whose own allocator owns the GPU's memory, or a
latency-bound loop that cannot afford an allocation or the synchronisation
of cudaFree).  It must produce exactly the state mickey_init_streams
produces, call after call, although every call reuses the same fixed array
inside the library.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1909_04750_gb300 import _native as N
from paper_1909_04750_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04750_gb300 import build as B
    B.build()
    return N.lib()


def _records(words, n):
    """Bitsliced state words [200, P] -> the 26-byte per-stream records of
    mickey_export_state (r0..r99 then s0..s99, MSB first)."""
    i = np.arange(n)
    bits = ((words[:, i // 32] >> (i % 32).astype(np.uint32)) & 1).astype(np.uint8)
    return np.concatenate([np.packbits(bits[:100].T, axis=1),
                           np.packbits(bits[100:].T, axis=1)], axis=1)


def _call(L, s, out, lens=True):
    keys = np.ascontiguousarray(s.keys, np.uint8)
    ivs = np.ascontiguousarray(s.ivs, np.uint8)
    lp = np.ascontiguousarray(s.iv_lens, np.uint32)
    return L.mickey_init_state_noalloc(keys.ctypes.data, ivs.ctypes.data,
                                       lp.ctypes.data if lens else None, s.n, out.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)


def _out(n):
    P = ((n + 31) // 32 + 31) // 32 * 32
    return torch.zeros((200, P), dtype=torch.int32, device="cuda")


def _noalloc(L, s, lens=True):
    out = _out(s.n)
    assert _call(L, s, out, lens) == N.OK
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def _regular(s, lens=True):
    from paper_1909_04750_gb300.streams import Streams
    st = Streams(s.keys, s.ivs, s.iv_lens if lens else None)
    rec, _ = st.export_state()
    st.free()
    return rec


def test_noalloc_equals_regular_init_two_calls_in_a_row(L):
    first = workloads.batched(5000)        # IV lengths 0..80 mixed within groups
    second = workloads.plain_scale(777)    # different size; array reused as is
    for s in (first, second):
        got = _records(_noalloc(L, s), s.n)
        assert np.array_equal(got, _regular(s))
    assert L.mickey_last_error() == N.OK


def test_noalloc_without_iv_lengths(L):
    # iv_lens = NULL: every IV is 80 bits and no lengths are copied
    s = workloads.batched(300)
    s.iv_lens[:] = 80
    got = _records(_noalloc(L, s, lens=False), s.n)
    assert np.array_equal(got, _regular(s, lens=False))


def test_noalloc_allocates_no_device_memory(L):
    # free device memory is the same before and after further calls (the
    # output buffer exists beforehand; the first call may load the module)
    s = workloads.batched(4000)
    out = _out(s.n)
    assert _call(L, s, out) == N.OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert _call(L, s, out) == N.OK
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    got = _records(out.cpu().numpy().view(np.uint32), s.n)
    assert np.array_equal(got, _regular(s))


def test_noalloc_rejects_bad_arguments(L):
    big = workloads.plain_scale(65537)
    state = torch.zeros(16, dtype=torch.int32, device="cuda")
    assert L.mickey_init_state_noalloc(big.keys.ctypes.data, big.ivs.ctypes.data, None, 65537,
                                       state.data_ptr(), None) == N.E_ARG
    assert L.mickey_last_error() == N.E_ARG
    s = workloads.plain_scale(40)
    lens = np.full(40, 80, np.uint32)
    lens[7] = 81
    assert L.mickey_init_state_noalloc(s.keys.ctypes.data, s.ivs.ctypes.data, lens.ctypes.data,
                                       40, state.data_ptr(), None) == N.E_IVLEN
    assert L.mickey_last_error() == N.E_IVLEN
    assert L.mickey_init_state_noalloc(None, s.ivs.ctypes.data, None, 40, state.data_ptr(),
                                       None) == N.E_ARG
