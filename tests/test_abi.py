"""The C ABI library on the CPU: it builds, loads without a GPU, exports every
symbol include/kq.h declares, and rejects invalid arguments before touching
the device."""
import ctypes as C

import numpy as np
import pytest

from paper_1101_0395_gb300 import kq

WS = C.c_void_p(1 << 20)  # aligned fake address: never dereferenced on these paths


def test_exports_every_declared_symbol():
    names = kq.exported_symbols()
    assert set(names) == {"kq_workspace_size", "kq_workspace_init", "kq_histogram", "kq_seed", "kq_lloyd", "kq_map",
                          "kq_lloyd_noalloc", "kq_status_read", "kq_status_clear", "kq_strerror",
                          "kq_batch_scratch_bytes", "kq_batch_workspace_size", "kq_batch_max_cluster",
                          "kq_batch_plan", "kq_batch_run", "kq_batch_tune", "kq_pixel_keys",
                          "kq_histogram_strided", "kq_set_wait_limit", "kq_map_ndc_read",
                          "kq_lab_points", "kq_seed_points", "kq_lloyd_points", "kq_lab_palette", "kq_map_labels",
                              "kq_live_bytes", "kq_live_init", "kq_live_reset", "kq_live_publish", "kq_live_done",
                              "kq_live_close", "kq_live_run"}
    L = kq.lib()
    for n in names:
        assert getattr(L, n) is not None


def test_workspace_size():
    small = kq.kq_workspace_size(1, 256)
    big = kq.kq_workspace_size(4096 * 4096, 256)
    assert small > (64 << 20) + (2 << 20)  # direct colour counters + presence bitmap
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
        assert L.kq_map(p, 10, p, K, p, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_seed(p, p, p, 8, 7, 1, None, p, WS, size, None) == kq.KQ_EINVAL  # USER is not a seeding scheme
    assert L.kq_seed(p, p, p, 8, -1, 1, None, p, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_seed(p, p, p, 8, 9, 1, None, p, WS, size, None) == kq.KQ_EINVAL
    bad = kq.SeedParams(1.0, 1e-4, 0, 0)
    assert L.kq_seed(p, p, p, 8, 1, 1, C.byref(bad), p, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_lloyd(p, p, p, 8, p, 1e-4, 0, 0, p, p, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_lloyd(p, p, p, 8, p, 1e-4, 10, 4, p, p, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_lloyd(p, p, p, 8, p, float("nan"), 10, 0, p, p, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_lloyd(None, p, p, 8, p, 1e-4, 10, 0, p, p, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_map(p, 10, p, 8, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_map(p, 10, None, 8, p, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_status_read(None, None, None) == kq.KQ_EINVAL
    assert L.kq_set_wait_limit(None, size, 1000, 1, None) == kq.KQ_EINVAL
    assert L.kq_map_ndc_read(None, None, None) == kq.KQ_EINVAL
    # the L*a*b* entry points
    assert L.kq_lab_points(None, p, p, None) == kq.KQ_EINVAL
    assert L.kq_seed_points(p, p, 8, 6, 1, p, None) == kq.KQ_EINVAL  # Forgy only
    assert L.kq_seed_points(p, p, 0, 0, 1, p, None) == kq.KQ_EINVAL
    assert L.kq_lloyd_points(p, p, p, 257, p, 1e-4, 10, 0, p, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_lloyd_points(p, p, p, 8, p, 1e-4, 0, 0, p, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_lloyd_points(p, p, p, 8, p, 1e-4, 10, 0, None, None, None, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_lab_palette(p, 0, p, None) == kq.KQ_EINVAL
    assert L.kq_map_labels(p, 10, p, p, None, p, WS, size, None) == kq.KQ_EINVAL
    assert L.kq_map_labels(p, 10, p, p, p, p, WS, 4096, None) == kq.KQ_EINVAL
    assert L.kq_set_wait_limit(WS, 4096, 1000, 1, None) == kq.KQ_EINVAL
    assert L.kq_workspace_init(None, size, None) == kq.KQ_EINVAL


def test_strerror():
    for code in (0, -1, -2, -3, -4, -5):
        assert kq.strerror(code) and kq.strerror(code) != "unknown status"
    assert kq.strerror(99) == "unknown status"


def _fake_items(spec):
    items = np.zeros(len(spec), dtype=kq.BATCH_ITEM_DTYPE)
    for i, (n, K) in enumerate(spec):
        for f in ("rgb", "idx", "keys", "weights", "labels", "scratch", "centers", "palette", "result"):
            items[i][f] = (1 << 20) + 4096 * i  # aligned; never dereferenced by the planner
        items[i]["n_pixels"], items[i]["K"], items[i]["scheme"] = n, K, 6
        items[i]["max_iter"], items[i]["capacity"], items[i]["eps"] = 100, n, 1e-4
        items[i]["lbg_max_iter"] = 100
    return items


def test_batch_structs_and_scratch():
    assert kq.BATCH_ITEM_DTYPE.itemsize == 136 and kq.BATCH_RESULT_DTYPE.itemsize == 96
    assert kq.BATCH_RESULT_DTYPE.itemsize == __import__('paper_1101_0395_gb300.serve', fromlist=['x']).RESULT_BYTES
    assert kq.kq_batch_scratch_bytes(1000) == 8192 + 16 * 9 + 256
    assert kq.kq_batch_scratch_bytes(0) == 272 and kq.kq_batch_scratch_bytes(-1) == 0


def test_batch_planner_orders_largest_work_first():
    items = _fake_items([(100, 16), (5000, 256), (0, 8), (70000, 32)])
    order, nb = kq.kq_batch_plan(items, kq.BatchConfig(1, 0, 0))
    assert nb == 0 and list(order) == [3, 1, 0, 2]
    order, nb = kq.kq_batch_plan(items, kq.BatchConfig(4, 0, 1000))
    assert nb == 2 and list(order) == [3, 1, 0, 2]
    order, nb = kq.kq_batch_plan(items, kq.BatchConfig(4, 0, 6000))
    assert nb == 1 and list(order) == [3, 1, 0, 2]
    for field, value in (("K", 0), ("K", 257), ("scheme", 9), ("max_iter", 0), ("n_pixels", -1),
                         ("capacity", -1), ("keys", 0), ("keys", (1 << 20) + 8), ("scratch", (1 << 20) + 16)):
        bad = items.copy()
        bad[1][field] = value
        with pytest.raises(kq.KqError):
            kq.kq_batch_plan(bad, kq.BatchConfig(1, 0, 0))
    for cl in (0, 3, 32):
        with pytest.raises(kq.KqError):
            kq.kq_batch_plan(items, kq.BatchConfig(cl, 0, 0))


def test_batch_run_rejects_bad_arguments_on_the_host():
    L = kq.lib()
    p = C.c_void_p(1 << 20)
    cfg = kq.BatchConfig(1, 0, 0)
    size = 1 << 30
    assert L.kq_batch_run(p, 4, p, 5, C.byref(cfg), WS, size, None) == kq.KQ_EINVAL   # n_big > n_items
    assert L.kq_batch_run(p, 4, p, 1, C.byref(cfg), WS, size, None) == kq.KQ_EINVAL   # clusters off, n_big > 0
    assert L.kq_batch_run(p, 4, p, 0, C.byref(cfg), C.c_void_p((1 << 20) + 8), size, None) == kq.KQ_EINVAL
    assert L.kq_batch_run(None, 4, p, 0, C.byref(cfg), WS, size, None) == kq.KQ_EINVAL
    assert L.kq_batch_run(p, 4, p, 0, None, WS, size, None) == kq.KQ_EINVAL
    bad = kq.BatchConfig(6, 0, 0)
    assert L.kq_batch_run(p, 4, p, 0, C.byref(bad), WS, size, None) == kq.KQ_EINVAL
    assert L.kq_batch_tune(None, p, 4, p, None, None, None, WS, size, None) == kq.KQ_EINVAL
    size2 = kq.kq_workspace_size(1000, 256)
    assert L.kq_histogram_strided(p, 10, 10, 29, 2, p, p, 10, p, WS, size2, None) == kq.KQ_EINVAL  # pitch < 3 w
    assert L.kq_histogram_strided(p, 10, 10, 30, 0, p, p, 10, p, WS, size2, None) == kq.KQ_EINVAL  # stride 0
    assert L.kq_histogram_strided(None, 10, 10, 30, 2, p, p, 10, p, WS, size2, None) == kq.KQ_EINVAL
    assert L.kq_pixel_keys(None, 10, p, None, None, None) == kq.KQ_EINVAL
    assert L.kq_pixel_keys(p, -1, p, None, None, None) == kq.KQ_EINVAL
    assert L.kq_pixel_keys(p, 1 << 31, p, None, None, None) == kq.KQ_EINVAL
