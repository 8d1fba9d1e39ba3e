"""The benchmark workloads at full size, checked against the oracle.

At these sizes the oracle evaluates sampled output elements one by one
(oracle_permute_sample, or the gather / interlace definitions on a subset of
indices), and properties that hold at any size are checked on the whole
output on the device: a permute followed by its inverse, interlace followed by
de-interlace and a reorder followed by its inverse give back the input bit for
bit.  The launch configuration is the one bench.py times (single calls on one
stream).
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import sync

pytestmark = pytest.mark.gpu

N_SAMPLES = 1 << 16


@pytest.fixture(scope="module")
def lr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1011_3583_gb300 import build, librearr
    build.build()
    librearr.load()
    return librearr


@pytest.fixture(scope="module")
def orc():
    return oracle.get()


def dev_from_np(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1).view(np.uint8)).to("cuda")


def sampled_equal(dev_out, e, lin: np.ndarray, want: np.ndarray) -> bool:
    import torch
    rows = dev_out.view(-1, e)[torch.from_numpy(lin).to("cuda")]
    return np.array_equal(rows.cpu().numpy().reshape(-1), want)


def inverse(perm):
    inv = [0] * len(perm)
    for i, p in enumerate(perm):
        inv[p] = i
    return inv


def permute_all_orders(lr, orc, dims, e, seed, orders=None):
    import torch
    n = int(np.prod(dims))
    src_np = synth.random_elements(seed, n * 1, e)
    src = dev_from_np(src_np)
    out = torch.empty_like(src)
    back = torch.empty_like(src)
    g = synth.rng(seed + 1)
    for perm in orders or itertools.permutations(range(len(dims))):
        perm = list(perm)
        out.fill_(0)
        lr.permute(out, src, e, dims, perm)
        lin = g.integers(0, n, size=N_SAMPLES, dtype=np.int64)
        lin[:4] = [0, n - 1, n // 2, 1]
        want = orc.permute_sample(src_np, e, dims, perm, lin)
        sync()
        assert sampled_equal(out, e, lin, want), (dims, perm, e)
        lr.permute(back, out, e, [dims[p] for p in perm], inverse(perm))
        sync()
        assert torch.equal(back, src), ("inverse round trip", dims, perm, e)


def test_config_transpose_1024(lr, orc):
    """1024 x 1024 fp32 transpose, compared in full."""
    import torch
    src_np = synth.random_elements(2024, 1024 * 1024, 4)
    src = dev_from_np(src_np)
    out = torch.empty_like(src)
    lr.permute(out, src, 4, [1024, 1024], [1, 0])
    sync()
    assert np.array_equal(out.cpu().numpy(), orc.permute(src_np, 4, [1024, 1024], [1, 0]))


def test_config_rank3_512_cubed(lr, orc):
    permute_all_orders(lr, orc, [512, 512, 512], 4, seed=512)


@pytest.mark.parametrize("e", [2, 4, 8])
def test_config_rank4_all_orders(lr, orc, e):
    permute_all_orders(lr, orc, [64, 128, 256, 64], e, seed=64 + e)


@pytest.mark.parametrize("kind", ["random", "block4096"])
def test_config_reorder_2p28(lr, orc, kind):
    import torch
    n = 1 << 28
    src_np = synth.random_elements(28, n, 4)
    idx_np = (synth.random_permutation(29, n) if kind == "random"
              else synth.block_shuffled_permutation(30, n, 4096))
    src, idx = dev_from_np(src_np), dev_from_np(idx_np)
    out = torch.empty_like(src)
    lr.reorder(out, src, idx, n, 4)
    g = synth.rng(31)
    lin = g.integers(0, n, size=N_SAMPLES, dtype=np.int64)
    lin[:2] = [0, n - 1]
    want = orc.reorder_sample(src_np, idx_np, 4, lin)
    sync()
    assert sampled_equal(out, 4, lin, want)
    # reorder by the inverse permutation restores the input everywhere
    inv = torch.empty_like(idx)
    inv.view(torch.int32)[idx.view(torch.int32).long()] = torch.arange(n, dtype=torch.int32, device="cuda")
    back = torch.empty_like(src)
    lr.reorder(back, out, inv, n, 4)
    sync()
    assert torch.equal(back, src)


def interlace_roundtrip(lr, orc, k, n, e, seed):
    import torch
    planes_np = [synth.random_elements(seed + j, n, e) for j in range(k)]
    planes = [dev_from_np(p) for p in planes_np]
    inter = torch.empty(n * k * e, dtype=torch.uint8, device="cuda")
    lr.interlace(inter, planes, n, e)
    g = synth.rng(seed + 100)
    rec = g.integers(0, n, size=N_SAMPLES // k, dtype=np.int64)
    rec[:2] = [0, n - 1]
    want = orc.interlace([p.reshape(n, e)[rec].reshape(-1) for p in planes_np], rec.size, e)
    lin = (rec[:, None] * k + np.arange(k)[None, :]).reshape(-1)
    sync()
    assert sampled_equal(inter, e, lin, want), ("interlace", k, n, e)
    outs = [torch.empty_like(p) for p in planes]
    lr.deinterlace(outs, inter, n, e)
    sync()
    for o, p in zip(outs, planes):
        assert torch.equal(o, p), ("de-interlace round trip", k, n, e)


def test_config_complex_split_2p28(lr, orc):
    """complex64 of 2^28 elements <-> real and imaginary fp32 planes."""
    import torch
    n = 1 << 28
    z_np = synth.random_elements(64, n, 8)
    z = dev_from_np(z_np)
    re, im = torch.empty(n * 4, dtype=torch.uint8, device="cuda"), torch.empty(n * 4, dtype=torch.uint8, device="cuda")
    lr.deinterlace([re, im], z, n, 4)
    g = synth.rng(65)
    rec = g.integers(0, n, size=N_SAMPLES, dtype=np.int64)
    sub = z_np.reshape(n, 8)[rec].reshape(-1)
    w_re, w_im = orc.deinterlace(sub, 2, rec.size, 4)
    sync()
    assert sampled_equal(re, 4, rec, w_re) and sampled_equal(im, 4, rec, w_im)
    back = torch.empty_like(z)
    lr.interlace(back, [re, im], n, 4)
    sync()
    assert torch.equal(back, z)


@pytest.mark.parametrize("k", [3, 4])
def test_config_image_planes_4096(lr, orc, k):
    """4096 x 4096 uint8 images, k planes, compared in full."""
    import torch
    n = 4096 * 4096
    planes_np = [synth.random_elements(70 + j, n, 1) for j in range(k)]
    planes = [dev_from_np(p) for p in planes_np]
    inter = torch.empty(n * k, dtype=torch.uint8, device="cuda")
    lr.interlace(inter, planes, n, 1)
    sync()
    assert np.array_equal(inter.cpu().numpy(), orc.interlace(planes_np, n, 1))
    outs = [torch.empty_like(p) for p in planes]
    lr.deinterlace(outs, inter, n, 1)
    sync()
    for o, p in zip(outs, planes_np):
        assert np.array_equal(o.cpu().numpy(), p)


@pytest.mark.parametrize("k", [2, 3, 4, 8])
def test_config_aos_soa_2p26(lr, orc, k):
    interlace_roundtrip(lr, orc, k, 1 << 26, 4, seed=80 + k)
