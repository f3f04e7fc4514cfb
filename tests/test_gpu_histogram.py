"""kq_histogram vs the oracle: bit-exact unique colours and weights."""
import numpy as np
import pytest
import torch

import oracle
from paper_1101_0395_gb300 import kq, synth
from tests.gpu_helpers import Run, new_ws, require_cuda, to_dev, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()


@pytest.mark.parametrize("name", ["plain_256", "paper_512"])
def test_histogram_workloads(name):
    img = synth.WORKLOADS[name].make(0)
    r = Run(img)
    keys, w = r.histogram()
    ok, ow = oracle.histogram(img)
    assert np.array_equal(keys, ok) and np.array_equal(w, ow)
    assert r.status() == kq.KQ_OK


@pytest.mark.parametrize("n", [1, 2, 15, 16, 17, 31, 33, 1000, 65537, 1000003])
def test_histogram_ragged_sizes(n):
    rng = np.random.default_rng(n)
    img = rng.integers(0, 256, size=(n, 3), dtype=np.uint8)
    img[n // 2:] = img[: n - n // 2] // 4 * 4  # repeats as well as singletons
    r = Run(img)
    keys, w = r.histogram()
    ok, ow = oracle.histogram(img)
    assert np.array_equal(keys, ok) and np.array_equal(w, ow)


@pytest.mark.parametrize("offset", [1, 3, 5, 8, 13, 15])
def test_histogram_misaligned_input(offset):
    img = synth.image(61, 47, 5, 12.0, 4.0, 900 + offset)
    flat = img.reshape(-1)
    buf = torch.zeros(flat.size + 64, dtype=torch.uint8, device="cuda")
    buf[offset:offset + flat.size] = to_dev(flat)
    r = Run(img)
    kq.kq_histogram(buf[offset:offset + flat.size], r.keys, r.weights, r.n_unique, r.ws)
    torch.cuda.synchronize()
    nu = int(r.n_unique.item())
    ok, ow = oracle.histogram(img)
    assert np.array_equal(u32(r.keys[:nu]), ok) and np.array_equal(u32(r.weights[:nu]), ow)


def test_histogram_every_colour_and_table_reset():
    k = np.arange(1 << 24, dtype=np.uint32)
    np.random.default_rng(7).shuffle(k)
    img = np.stack([(k >> 16) & 255, (k >> 8) & 255, k & 255], axis=1).astype(np.uint8)
    r = Run(img)
    keys, w = r.histogram()
    assert keys.size == 1 << 24 and np.array_equal(keys, np.arange(1 << 24, dtype=np.uint32)) and np.all(w == 1)
    # the tables were zeroed again: a second image on the same workspace is unaffected
    small = synth.WORKLOADS["plain_256"].make(1)
    r2 = Run(small, ws=r.ws)
    keys2, w2 = r2.histogram()
    ok, ow = oracle.histogram(small)
    assert np.array_equal(keys2, ok) and np.array_equal(w2, ow)


def test_histogram_repeat_same_workspace():
    img = synth.WORKLOADS["plain_256"].make(2)
    r = Run(img)
    a = r.histogram()
    b = r.histogram()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    ws_bytes = r.ws.numel()
    # counters and bitmap are back to zero after the call
    tables = r.ws[4096:4096 + (1 << 26) + (1 << 21)]
    assert int(tables.count_nonzero().item()) == 0
    assert ws_bytes == kq.kq_workspace_size(img.size // 3, 256)


def test_histogram_degenerate_inputs():
    r = Run(np.full((40, 3), 77, dtype=np.uint8))
    keys, w = r.histogram()
    assert keys.tolist() == [(77 << 16) | (77 << 8) | 77] and w.tolist() == [40]
    ws = new_ws(16)
    keys_t = torch.zeros(4, dtype=torch.int32, device="cuda")
    n_u = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    kq.kq_histogram(torch.zeros(0, dtype=torch.uint8, device="cuda"), keys_t, keys_t.clone(), n_u, ws, n_pixels=0)
    torch.cuda.synchronize()
    assert int(n_u.item()) == 0


def test_histogram_capacity_overflow():
    img = synth.WORKLOADS["plain_256"].make(0)
    ok, ow = oracle.histogram(img)
    cap = ok.size // 3
    r = Run(img, capacity=cap)
    keys, w = r.histogram()
    assert keys.size == cap
    assert np.array_equal(keys, ok[:cap]) and np.array_equal(w, ow[:cap])
    assert r.status() == kq.KQ_ECAPACITY
    kq.kq_status_clear(r.ws)
    assert r.status() == kq.KQ_OK


def test_histogram_invalid_arguments():
    ws = new_ws(16)
    t = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(kq.KqError) as e:
        kq.kq_histogram(torch.zeros(48, dtype=torch.uint8, device="cuda"), t, t, t[:1], ws[:1024])
    assert e.value.status == kq.KQ_EINVAL


@pytest.mark.parametrize("h,w,stride,pad", [(101, 77, 2, 0), (64, 64, 2, 5), (37, 90, 3, 2), (50, 51, 1, 0),
                                            (1, 1, 2, 0), (0, 10, 2, 0)])
def test_strided_histogram_matches_oracle_on_the_subsample(h, w, stride, pad):
    """Section 2.2's 2:1 subsampling: the histogram of the pixels (x, y) with x, y
    multiples of the stride, here with rows `pad` pixels longer than the image."""
    require_cuda()
    img = synth.image(max(h, 1), w + pad, 6, 12.0, 5.0, 77 + h)[:h] if h else np.zeros((0, w + pad, 3), np.uint8)
    pitch = 3 * (w + pad)
    sub = img[::stride, :w:stride]
    keys_o, w_o = oracle.histogram(sub.reshape(-1, 3)) if sub.size else (np.zeros(0, np.uint32),) * 2
    cap = max(1, h * w)
    keys = torch.zeros(cap, dtype=torch.int32, device="cuda")
    wts = torch.zeros(cap, dtype=torch.int32, device="cuda")
    nu = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.zeros(kq.kq_workspace_size(cap, 256), dtype=torch.uint8, device="cuda")
    rgb = to_dev(np.ascontiguousarray(img).reshape(-1)) if img.size else torch.zeros(1, dtype=torch.uint8,
                                                                                      device="cuda")
    kq.kq_histogram_strided(rgb, h, w, stride, keys, wts, nu, ws, pitch=pitch)
    torch.cuda.synchronize()
    n = int(nu.item())
    assert n == keys_o.size
    assert np.array_equal(u32(keys[:n]), keys_o) and np.array_equal(u32(wts[:n]), w_o)
    assert int(u32(wts[:n]).sum()) == ((h + stride - 1) // stride) * ((w + stride - 1) // stride)



@pytest.mark.parametrize("offset", [0, 7])
def test_large_misaligned_and_capacity(offset):
    # a misaligned 2^22 + 13 pixel image (head and tail pixels outside the 16-pixel
    # groups) with many singleton colours, twice on one workspace, then with room
    # for only a third of its colours
    rng = np.random.default_rng(4242 + offset)
    n = (1 << 22) + 13
    base = synth.WORKLOADS["paper_512"].make(5).reshape(-1, 3)
    img = base[rng.integers(0, base.shape[0], size=n)]
    img[: n // 5] = rng.integers(0, 256, size=(n // 5, 3), dtype=np.uint8)
    ok, ow = oracle.histogram(img)
    buf = torch.zeros(3 * n + 64, dtype=torch.uint8, device="cuda")
    buf[offset:offset + 3 * n] = to_dev(img.reshape(-1))
    r = Run(img)
    r.rgb = buf[offset:offset + 3 * n]
    keys, w = r.histogram()
    assert np.array_equal(keys, ok) and np.array_equal(w, ow)
    assert r.status() == kq.KQ_OK
    keys2, w2 = r.histogram()
    assert np.array_equal(keys2, ok) and np.array_equal(w2, ow)
    cap = ok.size // 3
    rc = Run(img, capacity=cap)
    kc, wc = rc.histogram()
    assert kc.size == cap and np.array_equal(kc, ok[:cap]) and np.array_equal(wc, ow[:cap])
    assert rc.status() == kq.KQ_ECAPACITY
