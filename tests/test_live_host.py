"""Host side of the live batch queue (kq_live_* in include/kq.h), without a GPU.

kq_live_init, kq_live_publish, kq_live_done and kq_live_close touch only host
memory, so an ordinary buffer stands in for the page-locked one here, and the
test writes the done marks that the running kernel would write."""
import ctypes as C

import numpy as np
import pytest

from paper_1101_0395_gb300 import kq

HEADER = 64
ITEM = kq.BATCH_ITEM_DTYPE.itemsize


def _queue(cap):
    L = kq.lib()
    nbytes = L.kq_live_bytes(cap)
    assert nbytes == HEADER + 2 * cap * (ITEM + 4)
    buf = np.full(nbytes, 0xAB, dtype=np.uint8)  # kq_live_init must clear it
    assert L.kq_live_init(buf.ctypes.data, cap) == kq.KQ_OK
    return L, buf


def _item(n=100, K=8):
    it = np.zeros(1, dtype=kq.BATCH_ITEM_DTYPE)
    for name in ("rgb", "idx", "labels", "centers", "palette", "result"):
        it[0][name] = 0x1000
    for name in ("keys", "weights"):
        it[0][name] = 0x2000
    it[0]["scratch"] = 0x3000
    it[0]["n_pixels"], it[0]["K"], it[0]["scheme"], it[0]["max_iter"] = n, K, kq.INIT["KPP"], 10
    it[0]["capacity"] = n
    return it


def _publish(L, buf, cls, it):
    seq = C.c_int64(-7)
    st = L.kq_live_publish(buf.ctypes.data, cls, it.ctypes.data, C.byref(seq))
    return st, seq.value


def _done_flags(buf, cap):
    return buf[HEADER + 2 * cap * ITEM:].view(np.uint32).reshape(2, cap)


def test_live_bytes_and_init():
    L = kq.lib()
    assert L.kq_live_bytes(0) == 0 and L.kq_live_bytes(-3) == 0
    L, buf = _queue(5)
    hdr = buf[:HEADER].view(np.uint32)
    assert hdr[0] == 0 and hdr[1] == 0 and hdr[2] == 0 and hdr[3] == 5
    assert not buf[HEADER:].any()
    assert L.kq_live_init(buf.ctypes.data, 0) == kq.KQ_EINVAL


def test_publish_sequence_ring_and_done():
    cap = 3
    L, buf = _queue(cap)
    items = buf[HEADER:HEADER + 2 * cap * ITEM].view(kq.BATCH_ITEM_DTYPE).reshape(2, cap)
    done = _done_flags(buf, cap)
    it = _item()
    seqs = []
    for j in range(cap):
        it[0]["seed"] = j
        st, seq = _publish(L, buf, 1, it)
        assert st == kq.KQ_OK and seq == j
        seqs.append(seq)
        assert items[1][j]["seed"] == j  # the copy sits in slot seq % cap of class 1
    assert tuple(buf[:8].view(np.uint32)) == (0, cap)
    # the ring is full until the item in slot 0 (seq 0) is done
    st, _ = _publish(L, buf, 1, it)
    assert st == kq.KQ_ECAPACITY
    assert L.kq_live_done(buf.ctypes.data, 1, 0) == 0
    done[1][0] = 1  # what the kernel writes for seq 0: seq + 1
    assert L.kq_live_done(buf.ctypes.data, 1, 0) == 1
    it[0]["seed"] = 77
    st, seq = _publish(L, buf, 1, it)
    assert st == kq.KQ_OK and seq == cap and items[1][0]["seed"] == 77
    # the slot's mark was cleared: seq 0 is gone, seq 3 not yet done
    assert L.kq_live_done(buf.ctypes.data, 1, cap) == 0 and done[1][0] == 0
    done[1][0] = cap + 1
    assert L.kq_live_done(buf.ctypes.data, 1, cap) == 1
    # class 0 has its own ring and counter
    st, seq = _publish(L, buf, 0, it)
    assert st == kq.KQ_OK and seq == 0
    assert tuple(buf[:8].view(np.uint32)) == (1, cap + 1)


def test_publish_rejects_bad_arguments_and_closed_queue():
    L, buf = _queue(4)
    it = _item()
    assert _publish(L, buf, 2, it)[0] == kq.KQ_EINVAL
    bad = it.copy()
    bad[0]["K"] = 0
    assert _publish(L, buf, 1, bad)[0] == kq.KQ_EINVAL
    bad = it.copy()
    bad[0]["keys"] = 0x2004  # not 16-byte aligned
    assert _publish(L, buf, 1, bad)[0] == kq.KQ_EINVAL
    assert tuple(buf[:8].view(np.uint32)) == (0, 0)
    assert L.kq_live_close(buf.ctypes.data) == kq.KQ_OK
    assert buf[8:12].view(np.uint32)[0] == 1
    assert _publish(L, buf, 1, it)[0] == kq.KQ_EINVAL
    assert L.kq_live_done(buf.ctypes.data, 1, 0) == 0
    assert L.kq_live_done(buf.ctypes.data, 1, -1) == 0


def test_run_rejects_bad_arguments():
    # checked before any CUDA call: no workspace, an idle limit of 0, a bad cluster size
    L, buf = _queue(2)
    ws = np.zeros(4096, dtype=np.uint8)
    assert L.kq_live_run(buf.ctypes.data, C.byref(kq.BatchConfig(1, 0, 0)), 1000, None, 0, None) == kq.KQ_EINVAL
    assert L.kq_live_run(buf.ctypes.data, C.byref(kq.BatchConfig(1, 0, 0)), 0, ws.ctypes.data, ws.size,
                         None) == kq.KQ_EINVAL
    assert L.kq_live_run(buf.ctypes.data, C.byref(kq.BatchConfig(3, 0, 0)), 1000, ws.ctypes.data, ws.size,
                         None) == kq.KQ_EINVAL
