"""The integer-pipe FP64 <-> FP32 conversions of the solver kernels (d2f_rn, d2f_rn2, f2d in
csrc/common.cuh) against the hardware conversions, bit for bit, on the GPU.

IEEE 754 fixes both results (binary64 -> binary32 round to nearest, ties to even; binary32 ->
binary64 exact), so the hardware conversion is the reference.  The inputs are 2^24 random bit
patterns (every exponent: zeros, subnormals, infinities and NaNs included) and, for 2^24 random
normal floats, the exact midpoints between neighbouring floats and the doubles one step either
side of them (the ties and near-ties of the rounding), and 2^24 products v 2^k rounded from
their exponent-shifted bits."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2402_13677_gb300", "csrc")
INCLUDE = os.path.join(HERE, "..", "include")

SRC = r'''
#include <cstdio>
#include "common.cuh"
using namespace ebit;

__device__ unsigned long long mix(unsigned long long z) {   // splitmix64 finaliser
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_check(long long n, unsigned long long* bad) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    unsigned long long r = mix((unsigned long long)t);
    unsigned long long cnt = 0;
    // a random bit pattern
    double v = __longlong_as_double((long long)r);
    float a = d2f_rn(v), b = __double2float_rn(v);
    if (__float_as_uint(a) != __float_as_uint(b) && !(a != a && b != b)) ++cnt;
    // ties and near-ties: a random normal float f and the midpoint to its successor
    unsigned u = (unsigned)(mix(r) >> 32);
    unsigned e = (u >> 23) & 0xffu;
    if (e >= 1u && e <= 253u) {
        float f = __uint_as_float(u), g = __uint_as_float(u + 1u);
        double mid = 0.5 * ((double)f + (double)g);
        long long mb = __double_as_longlong(mid);
        for (int d = -1; d <= 1; ++d) {
            double w = __longlong_as_double(mb + d);
            float x = d2f_rn(w), y = __double2float_rn(w);
            if (__float_as_uint(x) != __float_as_uint(y)) ++cnt;
        }
    }
    // scaled rounding: v 2^k, v a random normal binary64 with exponent in [-200, 200) and k in
    // [-160, 160], so that v 2^k (exact in binary64) is normal
    {
        int k = (int)(mix(r ^ 0x5bd1e995ull) % 321ull) - 160;
        long long ev = 1023 + (long long)(mix(r + 7ull) % 400ull) - 200;
        double vs = __longlong_as_double((long long)(mix(r + 9ull) & 0x800fffffffffffffull) | (ev << 52));
        double p2 = __longlong_as_double((long long)(1023 + k) << 52);
        float x2 = d2f_rn2(vs, k), y2 = __double2float_rn(vs * p2);
        if (__float_as_uint(x2) != __float_as_uint(y2)) ++cnt;
    }
    // widening: a random bit pattern as a float
    float h = __uint_as_float((unsigned)r);
    double p = f2d(h), q = (double)h;
    if (__double_as_longlong(p) != __double_as_longlong(q) && !(p != p && q != q)) ++cnt;
    if (cnt) atomicAdd(bad, cnt);
}

int main() {
    unsigned long long* bad;
    cudaMalloc(&bad, sizeof(unsigned long long));
    cudaMemset(bad, 0, sizeof(unsigned long long));
    long long n = 1LL << 24;
    k_check<<<(unsigned)((n + 255) / 256), 256>>>(n, bad);
    unsigned long long h = 0;
    cudaError_t err = cudaMemcpy(&h, bad, sizeof(h), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) { printf("cuda error %s\n", cudaGetErrorString(err)); return 2; }
    printf("mismatches %llu\n", h);
    return 0;
}
'''


def test_integer_pipe_conversions_match_the_hardware(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "conv.cu"
    src.write_text(SRC)
    exe = tmp_path / "conv"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC, "-I",
                    INCLUDE, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout
    assert "mismatches 0" in out, out
