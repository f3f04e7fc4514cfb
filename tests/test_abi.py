"""The C ABI library on the CPU: it builds, loads without a GPU, exports every
symbol include/kq.h declares, and rejects invalid arguments before touching
the device."""
import ctypes as C

from paper_1101_0395_gb300 import kq

WS = C.c_void_p(1 << 20)  # aligned fake address: never dereferenced on these paths


def test_exports_every_declared_symbol():
    names = kq.exported_symbols()
    assert set(names) == {"kq_workspace_size", "kq_workspace_init", "kq_histogram", "kq_seed", "kq_lloyd", "kq_map",
                          "kq_lloyd_noalloc", "kq_status_read", "kq_status_clear", "kq_strerror"}
    L = kq.lib()
    for n in names:
        assert getattr(L, n) is not None


def test_workspace_size():
    small = kq.kq_workspace_size(1, 256)
    big = kq.kq_workspace_size(4096 * 4096, 256)
    assert small > (64 << 20) + (16 << 20)  # direct colour tables + lookup table
    assert big - small >= 9 * (4096 * 4096 - 1) - 1024  # 9 bytes per possible unique colour
    assert kq.kq_workspace_size(1 << 30, 256) == kq.kq_workspace_size(1 << 24, 256)  # N' <= 2^24
    assert kq.kq_workspace_size(-1, 256) == 0 and kq.kq_workspace_size(10, 0) == 0
    assert kq.kq_workspace_size(10, 257) == 0


def test_invalid_arguments_are_rejected_synchronously():
    L = kq.lib()
    size = kq.kq_workspace_size(1000, 256)
    p = C.c_void_p(1 << 20)
    # null or misaligned workspace, too small a workspace
    assert L.kq_histogram(p, 10, p, p, 10, p, None, size, None) == kq.KQ_EINVAL
    assert L.kq_histogram(p, 10, p, p, 10, p, C.c_void_p((1 << 20) + 8), size, None) == kq.KQ_EINVAL
    assert L.kq_histogram(p, 10, p, p, 10, p, WS, 4096, None) == kq.KQ_EINVAL
    assert L.kq_histogram(p, -1, p, p, 10, p, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_histogram(None, 10, p, p, 10, p, WS, size, None) == kq.KQ_EINVAL
    # K out of range, bad scheme, bad flags, bad iteration limit
    for K in (0, 257):
        assert L.kq_seed(p, p, p, K, 0, 1, None, p, WS, size, None) == kq.KQ_EINVAL
        assert L.kq_lloyd(p, p, p, K, p, 1e-4, 10, 0, p, p, None, None, WS, size, None) == kq.KQ_EINVAL
        assert L.kq_map(p, 10, p, p, p, p, K, p, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_seed(p, p, p, 8, 7, 1, None, p, WS, size, None) == kq.KQ_EINVAL  # USER is not a seeding scheme
    assert L.kq_seed(p, p, p, 8, -1, 1, None, p, WS, size, None) == kq.KQ_EINVAL
    bad = kq.SeedParams(1.0, 1e-4, 0, 0)
    assert L.kq_seed(p, p, p, 8, 1, 1, C.byref(bad), p, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_lloyd(p, p, p, 8, p, 1e-4, 0, 0, p, p, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_lloyd(p, p, p, 8, p, 1e-4, 10, 4, p, p, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_lloyd(p, p, p, 8, p, float("nan"), 10, 0, p, p, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_lloyd(None, p, p, 8, p, 1e-4, 10, 0, p, p, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_map(p, 10, p, p, p, p, 8, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_status_read(None, None, None) == kq.KQ_EINVAL
    assert L.kq_workspace_init(None, size, None) == kq.KQ_EINVAL


def test_strerror():
    for code in (0, -1, -2, -3, -4, -5):
        assert kq.strerror(code) and kq.strerror(code) != "unknown status"
    assert kq.strerror(99) == "unknown status"
