"""The bit-packed layout of host pages (the encoder tp_table_append uses),
checked on the CPU through tp_debug_pack_bits against the layout the header
states, written out bit by bit here: value i occupies stream bits
[i * bits, (i + 1) * bits), least significant first, and stream bit j is bit
j % 32 of word j / 32.  No GPU is needed; the device decoder of the same
layout is covered by the GPU parity tests of paged tables."""
import ctypes

import numpy as np
import pytest

from paper_2508_05029_gb300 import build, theseus


@pytest.fixture(scope="module")
def lib():
    build.build()
    lib = theseus.load()
    return lib


def _pack(lib, values, bits):
    v = np.ascontiguousarray(values, dtype=np.uint64)
    words = np.full((len(v) * bits + 31) // 32 + 1, 0xDEADBEEF, dtype=np.uint32)   # +1: a guard word
    rc = lib.tp_debug_pack_bits(v.ctypes.data_as(ctypes.c_void_p), len(v), bits,
                                words.ctypes.data_as(ctypes.c_void_p))
    return rc, words


def _layout(values, bits):
    """The stated layout, one stream bit at a time."""
    n_words = (len(values) * bits + 31) // 32
    words = [0] * n_words
    for i, x in enumerate(int(v) for v in values):
        for b in range(bits):
            if (x >> b) & 1:
                j = i * bits + b
                words[j // 32] |= 1 << (j % 32)
    return words


@pytest.mark.parametrize("bits", list(range(1, 32)))
def test_every_width_matches_the_stated_layout(lib, bits):
    rng = np.random.default_rng(bits)
    for n in (0, 1, 31, 32, 33, 97, 1000):
        values = rng.integers(0, 1 << bits, n, dtype=np.uint64)
        if n:
            values[-1] = (1 << bits) - 1          # the widest value at the ragged end
        rc, words = _pack(lib, values, bits)
        assert rc == theseus.TP_OK
        n_words = (n * bits + 31) // 32
        assert words[:n_words].tolist() == _layout(values, bits)
        assert words[n_words] == 0xDEADBEEF      # nothing written past the stream


@pytest.mark.parametrize("bits", [1, 5, 12, 21, 31])
def test_values_read_back_from_the_stream(lib, bits):
    rng = np.random.default_rng(100 + bits)
    values = rng.integers(0, 1 << bits, 777, dtype=np.uint64)
    _, words = _pack(lib, values, bits)
    stream = int.from_bytes(words.astype("<u4").tobytes(), "little")
    back = [(stream >> (i * bits)) & ((1 << bits) - 1) for i in range(len(values))]
    assert back == values.tolist()


def test_refusals(lib):
    assert _pack(lib, [1 << 5], 5)[0] == theseus.TP_E_INVALID      # does not fit
    assert _pack(lib, [0], 0)[0] == theseus.TP_E_INVALID           # bits out of range
    assert _pack(lib, [0], 32)[0] == theseus.TP_E_INVALID
