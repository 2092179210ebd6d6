"""The Philox-4x32-10 key/counter layout of the random-phase initial state
(Sec. 2: the paper draws its phases with cuRAND) against cuRAND's device API:
a generator set up with curand_init(seed, subsequence = site index, offset = 0)
yields, as its first four 32-bit outputs, the block function of the oracle at
key = seed, counter = (0, 0, site index).  The test compiles a small kernel that
calls cuRAND and compares words for sites spread over a 2048^3 index range.

The mapping of two words to a uniform double is this code's convention; the
test reports how cuRAND's curand_uniform_double compares, without asserting it."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

SRC = r'''
#include <curand_kernel.h>
__global__ void k(unsigned long long seed, const unsigned long long *idx, int n, uint4 *w, double *u)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t s;
    curand_init(seed, idx[i], 0, &s);
    w[i] = curand4(&s);
    curandStatePhilox4_32_10_t t;
    curand_init(seed, idx[i], 0, &t);
    u[i] = curand_uniform_double(&t);
}
extern "C" int curand_words(unsigned long long seed, const unsigned long long *idx, int n, unsigned *w, double *u)
{
    unsigned long long *d_idx = 0; uint4 *d_w = 0; double *d_u = 0;
    if (cudaMalloc(&d_idx, n * sizeof(*d_idx)) || cudaMalloc(&d_w, n * sizeof(uint4)) || cudaMalloc(&d_u, n * sizeof(double)))
        return 1;
    cudaMemcpy(d_idx, idx, n * sizeof(*d_idx), cudaMemcpyHostToDevice);
    k<<<(n + 127) / 128, 128>>>(seed, d_idx, n, d_w, d_u);
    cudaMemcpy(w, d_w, n * sizeof(uint4), cudaMemcpyDeviceToHost);
    cudaMemcpy(u, d_u, n * sizeof(double), cudaMemcpyDeviceToHost);
    const int err = cudaGetLastError() != cudaSuccess;
    cudaFree(d_idx); cudaFree(d_w); cudaFree(d_u);
    return err;
}
'''


def test_philox_layout_matches_curand(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    (tmp_path / "c.cu").write_text(SRC)
    so = tmp_path / "libc.so"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    str(tmp_path / "c.cu"), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    rng = np.random.Generator(np.random.PCG64(9))
    idx = np.concatenate([np.arange(8), rng.integers(0, 2048 ** 3, size=56)]).astype(np.uint64)
    for seed in (1, 3, 0x9E3779B97F4A7C15):
        w = np.zeros(4 * len(idx), dtype=np.uint32)
        u = np.zeros(len(idx), dtype=np.float64)
        assert lib.curand_words(ctypes.c_ulonglong(seed), idx.ctypes.data_as(ctypes.c_void_p), len(idx),
                                w.ctypes.data_as(ctypes.c_void_p), u.ctypes.data_as(ctypes.c_void_p)) == 0
        same_u = 0
        for i, s in enumerate(idx):
            s = int(s)
            ref = O.philox4x32_10((0, 0, s & 0xFFFFFFFF, s >> 32), (seed & 0xFFFFFFFF, seed >> 32))
            assert list(w[4 * i:4 * i + 4]) == ref, (seed, s)
            same_u += u[i] == O.site_uniform(seed, s)
        print("seed %#x: curand_uniform_double equals the oracle's uniform at %d of %d sites"
              % (seed, same_u, len(idx)))
