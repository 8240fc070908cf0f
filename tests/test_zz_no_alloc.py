"""The allocation-free Gram entry point, lobpcg_gram_noalloc.

Callers that cannot allocate device memory at the moment they need a Gram
(inside a framework that owns the memory pool, in a callback that runs under an
allocator lock, in a loop that must not synchronise the device through
cudaMalloc/cudaFree) use this entry point: it takes its scratch from a fixed
array inside the library.  Here it is called through the C ABI twice in a row
and compared with the allocating entry point lobpcg_gram (tensor-core mode)
and with the definition U^T V, within the same error bound as the kernel tests.

This file is collected last so that a failure here never hides another test.
"""
import numpy as np
import pytest

import synth
import paper_1704_07458_gb300 as gb
from gpu_util import torch_cuda, dev, host, gamma

pytestmark = pytest.mark.gpu


def _bound(U, V, slices, n):
    unit = 4 * (4 + 4 * slices) * 2.0 ** (-8 * slices)
    nck = (n + 63) // 64
    mu = np.stack([np.abs(U[64 * c:64 * c + 64]).max(0) for c in range(nck)])
    mv = np.stack([np.abs(V[64 * c:64 * c + 64]).max(0) for c in range(nck)])
    absg = np.abs(U).T @ np.abs(V)
    return 2 * gamma(n) * absg + unit * 64 * 4 * (mu.T @ mv) + 2.0 ** -44 * absg


def _pair(n, p, q, seed, slices):
    torch = torch_cuda()
    U = synth.normal_block(seed, 1, n, p) * np.logspace(-5, 1, p)[None, :]
    V = synth.normal_block(seed + 1, 1, n, q) * np.logspace(2, -4, q)[None, :]
    Ud, Vd = dev(U, p + 1), dev(V, q)
    G1 = dev(np.full(p * q, np.nan))
    G2 = dev(np.full(p * q, np.nan))
    assert gb.lobpcg_gram_noalloc(n, Ud, p + 1, p, Vd, q, q, G1, p, slices) == 0
    assert gb.lobpcg_gram(n, Ud, p + 1, p, Vd, q, q, G2, p, gb.LOBPCG_GEMM_OZAKI, slices) == 0
    torch.cuda.synchronize()
    g1 = host(G1).reshape(q, p).T
    g2 = host(G2).reshape(q, p).T
    return U, V, g1, g2


@pytest.mark.parametrize("slices", [6, 4])
def test_noalloc_gram_matches_allocating_entry_point_twice(slices):
    # first: a shape whose normal row split needs more scratch than the fixed
    # array holds (the variant uses fewer, longer slabs); second: a small one
    for (n, p, q, seed) in [(100000, 256, 256, 11), (4099, 71, 142, 12)]:
        U, V, g1, g2 = _pair(n, p, q, seed, slices)
        ref = U.T @ V
        b = _bound(U, V, slices, n)
        assert np.all(np.abs(g1 - ref) <= b)
        assert np.all(np.abs(g1 - g2) <= 2 * b)


def test_noalloc_gram_rejects_shapes_beyond_its_scratch():
    torch_cuda()
    # p * q * 16 bytes > 16 MiB: refused before any device work
    assert gb.lobpcg_gram_noalloc(10, 1, 2048, 2048, 1, 1024, 1024, 1, 2048, 0) == \
        gb.LOBPCG_ERR_ARG
