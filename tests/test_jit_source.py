"""The run-time compiled kernel source builds under NVRTC for sm_103a, for
shapes covering every branch of the shape struct (no GPU needed: NVRTC
compiles to a cubin on the host)."""
import ctypes
import os

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2508_05029_gb300", "csrc")
HEADERS = ["kernels.cuh", "device.cuh", "pipeline.cuh", "jit_common.cuh", "jit_dense.cuh", "jit_batch.cuh"]


def _nvrtc():
    for name in ("libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("NVRTC not available")


def _shape(filter=1, ftype=0, join=1, ktype=0, part=0, lip=0, many=0, groups=((0, 2, 2), (0, 2, 1), (1, 0, 5)),
           sums=((0, 1, 0, 1, 0), (1, 1, 1, 2, 1), (0, 1, 0, 1, 0)), fast=True, xjoins=(), gdim=(0, 0, 0, 0)):
    """groups: (side, type, bits); sums: (kind, atype, btype, mode, narrow);
    xjoins: further joins (kind, key type, lookahead); gdim: join of each dimension field."""
    def arr(name, vals, n):
        vals = list(vals) + [0] * (n - len(vals))
        return f"{name}[{n}] = {{{', '.join(map(str, vals))}}}"
    g = list(zip(*groups)) if groups else ((), (), ())
    s = list(zip(*sums)) if sums else ((), (), (), (), ())
    return ("struct JS {\n"
            f"  static constexpr int filter = {filter}, ftype = {ftype}, join = {join}, ktype = {ktype}, part = {part}, "
            f"lip = {lip}, many = {many};\n"
            f"  static constexpr int nx = {len(xjoins)}, {arr('xjoin', [x[0] for x in xjoins], 3)}, "
            f"{arr('xktype', [x[1] for x in xjoins], 3)}, {arr('xlip', [x[2] for x in xjoins], 3)};\n"
            f"  static constexpr int ng = {len(groups)}, {arr('gdim', gdim, 4)};\n"
            f"  static constexpr int {arr('gside', g[0], 4)}, {arr('gtype', g[1], 4)}, {arr('gbits', g[2], 4)};\n"
            f"  static constexpr int ns = {len(sums)};\n"
            f"  static constexpr int {arr('skind', s[0], 8)}, {arr('atype', s[1], 8)}, {arr('btype', s[2], 8)}, "
            f"{arr('mode', s[3], 8)}, {arr('narrow', s[4], 8)};\n"
            f"  static constexpr bool fast = {'true' if fast else 'false'}, lo_only = false;\n}};\n")


SHAPES = {
    "star-lowcard-direct": _shape(),
    "exact-128": _shape(fast=False, sums=((0, 1, 0, 0, 0), (1, 1, 1, 0, 0))),
    "hash32-partitioned": _shape(join=2, part=1),
    "hash64-i64-key": _shape(join=3, ktype=1),
    "no-filter-no-join": _shape(filter=0, join=0, groups=((0, 0, 4), (0, 1, 3)), sums=((0, 0, 0, 1, 0),)),
    "i64-filter-u8-wide-field": _shape(ftype=1, groups=((0, 2, 9), (1, 0, 3)), sums=((1, 0, 2, 2, 0),)),
    "count-only": _shape(sums=()),
    "lip-direct": _shape(lip=1),
    "lip-hash64-partitioned": _shape(join=3, ktype=1, part=1, lip=1),
    "fan-out-hash64": _shape(join=3, ktype=1, many=1),
    "star-three-further-joins": _shape(xjoins=((1, 0, 0), (2, 1, 1), (3, 1, 0)),
                                       groups=((1, 0, 3), (1, 0, 4), (1, 0, 2), (1, 0, 2)), gdim=(0, 1, 2, 3)),
}


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_nvrtc_compiles_shape(name):
    _compile(_nvrtc(), SHAPES[name] + '#include "jit_dense.cuh"\n')


def _compile(lib, source):
    texts = [open(os.path.join(CSRC, h)).read().encode() for h in HEADERS]
    names = [h.encode() for h in HEADERS]
    src = source.encode()
    prog = ctypes.c_void_p()
    n = len(HEADERS)
    arr_t = ctypes.c_char_p * n
    rc = lib.nvrtcCreateProgram(ctypes.byref(prog), src, b"tp_jit.cu", n, arr_t(*texts), arr_t(*names))
    assert rc == 0
    opts = [b"--gpu-architecture=sm_103a", b"-std=c++17", b"--device-int128",
            b"-DTP_ST_CONSUMERS=24", b"-DTP_ST_RPL=2", b"-DTP_ST_CTAS=1"]
    rc = lib.nvrtcCompileProgram(prog, len(opts), (ctypes.c_char_p * len(opts))(*opts))
    size = ctypes.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, ctypes.byref(size))
    log = ctypes.create_string_buffer(size.value)
    lib.nvrtcGetProgramLog(prog, log)
    cubin = ctypes.c_size_t()
    if rc == 0:
        lib.nvrtcGetCUBINSize(prog, ctypes.byref(cubin))
    lib.nvrtcDestroyProgram(ctypes.byref(prog))
    assert rc == 0, log.value.decode(errors="replace")[:2000]
    assert cubin.value > 0


def test_nvrtc_compiles_batch_kernel():
    """The batched queue kernel with two shapes (shared-memory 32-bit table;
    device-memory 64-bit low words) and the dispatcher the host writes."""
    lib = _nvrtc()
    a = _shape().replace("struct JS {", "struct JS_0 {")
    b = _shape(fast=False, join=2, sums=((0, 1, 0, 0, 0), (1, 1, 1, 0, 0))).replace("struct JS {", "struct JS_1 {")
    b = b.replace("lo_only = false", "lo_only = true")
    disp = ("__device__ void tpj::dispatch_probe(const tpk::BatchQuery& B, uint64_t r0, uint64_t r1, "
            "unsigned char* smem) {\n    switch (B.shape) {\n"
            "    case 0: probe_tile<JS_0>(B, r0, r1, smem); break;\n"
            "    case 1: probe_tile<JS_1>(B, r0, r1, smem); break;\n    default: break;\n    }\n}\n")
    _compile(lib, a + b + '#include "jit_batch.cuh"\n' + disp)
