"""The three loading paths of the init kernel against the scalar oracle.

Keys, IVs and IV lengths in their own order and 16-byte aligned are read
with 16-byte loads into registers (the last group, if partial, byte by
byte); unaligned they are copied into shared memory first; through the
batch planner's permutation each record is read byte by byte.  Every path
must give the same bitsliced inputs, so the keystream of every instance is
compared with the oracle's, exactly, for IV lengths mixed inside groups,
uniform but not a multiple of 4, zero, and absent (80 bits).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1909_04750_gb300 import _native as N
from paper_1909_04750_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04750_gb300 import build as B
    B.build()
    N.lib()


def _case(n, kind, seed):
    s = workloads.plain_scale(n)
    rng = np.random.default_rng(seed)
    if kind == "mixed":            # every length 0..80, mixed inside groups
        s.iv_lens[:] = rng.integers(0, 81, n)
    elif kind not in ("80", "none"):
        s.iv_lens[:] = int(kind)
    return s


def _ref(s, n_bits):
    return oracle.batch_bytes(s.keys, s.ivs, s.iv_lens, n_bits, threads=THREADS)


def _device(arr, offset, dtype=torch.uint8):
    """A CUDA tensor holding arr's bytes that starts `offset` bytes into its
    allocation (offset 0: 16-byte aligned)."""
    raw = np.frombuffer(np.ascontiguousarray(arr).tobytes(), np.uint8)
    buf = torch.zeros(raw.size + 64, dtype=torch.uint8, device="cuda")
    buf[offset:offset + raw.size] = torch.from_numpy(raw.copy()).cuda()
    t = buf[offset:offset + raw.size]
    return t.view(dtype) if dtype != torch.uint8 else t


def _streams(s, kind, key_off=0, iv_off=0, len_off=0):
    from paper_1909_04750_gb300.streams import Streams
    keys = _device(s.keys, key_off).view(s.n, 10)
    ivs = _device(s.ivs, iv_off).view(s.n, 10)
    lens = None if kind == "none" else _device(s.iv_lens.astype(np.int32), len_off, torch.int32)
    st = Streams(keys, ivs, lens)
    st._inputs = (keys, ivs, lens)
    return st


@pytest.mark.parametrize("kind", ["mixed", "80", "none", "37", "48", "0"])
@pytest.mark.parametrize("n", [32 * 300, 32 * 300 + 7, 5 * 1024 + 1])
def test_aligned_and_unaligned_inputs_every_instance(n, kind):
    s = _case(n, kind, n)
    ref = _ref(s, 96)
    outs = []
    for offs in ((0, 0, 0), (1, 0, 0), (0, 6, 4), (3, 5, 8)):
        if kind == "none" and offs[2]:
            continue
        st = _streams(s, kind, *offs)
        outs.append(st.generate(96, "bytes").cpu().numpy())
        st.sync()
    for got in outs:
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("n", [1000, 4099, 32 * 128 + 3])
def test_host_inputs_any_count(n):
    # host inputs are copied to 16-byte aligned offsets whatever n is
    from paper_1909_04750_gb300.streams import Streams
    s = _case(n, "mixed", 7 + n)
    st = Streams(s.keys, s.ivs, s.iv_lens)
    got = st.generate(200, "bytes").cpu().numpy()
    st.sync()
    assert np.array_equal(got, _ref(s, 200))
    # a reset with other inputs through the same staging buffer
    s2 = _case(n, "48", 9 + n)
    st.reset(s2.keys, s2.ivs, s2.iv_lens)
    got = st.generate(200, "bytes").cpu().numpy()
    st.sync()
    assert np.array_equal(got, _ref(s2, 200))


def test_full_size_mixed_lengths_sampled():
    # 2^20 instances with mixed IV lengths through the 16-byte loads
    s = _case(1 << 20, "mixed", 77)
    st = _streams(s, "mixed")
    out = st.generate(1024, "bytes")
    st.sync()
    rng = np.random.default_rng(5)
    rows = np.array(sorted(set(range(64)) | set(range(s.n - 64, s.n))
                           | set(rng.integers(0, s.n, 4096).tolist())))
    got = out[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.array_equal(got, _ref(s.subset(rows), 1024))
