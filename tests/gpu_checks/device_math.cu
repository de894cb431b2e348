// Checks of the library's device arithmetic (paper_2010_14244_gb300/csrc/gmp_device.cuh) against
// CUDA's own results: the reciprocal against __frcp_rn (every input the colony can produce), the
// roulette index against __umul64hi, the u32 -> f32 conversion against __uint2float_rn (every c < 2^29), Philox4x32-10 against cuRAND's curand_Philox4x32_10, the
// reciprocal modulo against %, and isqrt against a bit-by-bit root. Roulette weights are written out
// for the Python test to compare with the CPU oracle's exact quantisation.
//
// usage: device_math checks            -> "name mismatches" lines
//        device_math weights IN OUT    -> IN: u32 count, then per vector u32 n + n f32 scores
//                                         OUT: the u64 weights of every vector, in order
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include <cstdio>
#include <cstdlib>
#include <string_view>
#include <vector>

#include "gmp_device.cuh"

using namespace gmp;

__global__ void k_rcp(unsigned long long lo, unsigned long long n, unsigned long long* bad) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const float b = lo == 0 ? (float)(unsigned)(i + 1) : __uint_as_float((unsigned)(lo + i));
        if (__float_as_uint(rcp_rn(b)) != __float_as_uint(__frcp_rn(b))) atomicAdd(bad, 1ull);
    }
}

__global__ void k_cvt(unsigned long long* bad) {  // every c < 2^29
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < (1u << 29); c += gridDim.x * blockDim.x)
        if (__float_as_uint(u32_to_f32_rn(c)) != __float_as_uint(__uint2float_rn(c))) atomicAdd(bad, 1ull);
}

__device__ unsigned long long mix(unsigned long long x) {
    x ^= x >> 31;
    x *= 0x7FB5D329728EA185ull;
    x ^= x >> 27;
    x *= 0x81DADEF4BC2DD44Dull;
    return x ^ (x >> 33);
}

__global__ void k_misc(unsigned long long n, unsigned long long* bad) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long a = mix(i), b = mix(i + 0x9E3779B97F4A7C15ull);
        // roulette index, S < 2^32
        const uint32_t S = (uint32_t)(b >> (32 + (i % 32))) + (uint32_t)(i & 1);
        if ((unsigned long long)draw_index(a, S) != __umul64hi(a, (unsigned long long)S)) atomicAdd(bad + 0, 1ull);
        // Philox against cuRAND
        const uint4 c = make_uint4((unsigned)a, (unsigned)(a >> 32), (unsigned)b, (unsigned)(b >> 32));
        const uint4 x = philox4x32_10(c, (unsigned)(i * 2654435761u), (unsigned)(i >> 7));
        const uint4 y = curand_Philox4x32_10(c, make_uint2((unsigned)(i * 2654435761u), (unsigned)(i >> 7)));
        if (x.x != y.x || x.y != y.y || x.z != y.z || x.w != y.w) atomicAdd(bad + 1, 1ull);
        // reciprocal modulo, 1 <= d <= 2^24
        const unsigned xv = (unsigned)a, d = 1u + (unsigned)(b % (1ull << (1 + (i % 24))));
        if (mod_magic(xv, d, 0xFFFFFFFFu / d) != xv % d) atomicAdd(bad + 2, 1ull);
        // integer square root, n < 2^58
        const unsigned long long nn = b >> (6 + (i % 50));
        const unsigned long long r = isqrt_u64(nn);
        if (!(r * r <= nn && (r + 1) * (r + 1) > nn)) atomicAdd(bad + 3, 1ull);
        // float weights equal the integer-exponent weights
        const unsigned mbits = (unsigned)(a >> 33) & 0x7F7FFFFFu;  // any finite non-negative float
        const unsigned sbits = (unsigned)(b >> 33) % (mbits + 1u);  // s <= m
        if (roulette_weight_f(sbits, weight_scale(mbits)) != roulette_weight(sbits, mbits)) atomicAdd(bad + 4, 1ull);
    }
}

__global__ void k_weights(const unsigned* off, const unsigned* len, const float* s, unsigned long long* w,
                          unsigned nvec) {
    const unsigned v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvec) return;
    unsigned mb = 0;
    for (unsigned i = 0; i < len[v]; ++i) mb = max(mb, __float_as_uint(s[off[v] + i]));
    const WeightScale sc = weight_scale(mb);
    for (unsigned i = 0; i < len[v]; ++i) w[off[v] + i] = roulette_weight_f(__float_as_uint(s[off[v] + i]), sc);
}

// Non-integer-exponent arithmetic, one record per thread: log2_cw(x), exp2_sat(L), score_frac(tf, a, c, b).
struct FracIn {
    float x, L, tf, alpha;
    unsigned c;
    float beta;
};

__global__ void k_frac(const FracIn* in, float* out, unsigned n) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const FracIn r = in[i];
    out[3 * (size_t)i] = log2_cw(r.x);
    out[3 * (size_t)i + 1] = exp2_sat(r.L);
    out[3 * (size_t)i + 2] = score_frac(r.tf, r.alpha, r.c, r.beta);
}

static int frac(const char* in, const char* out) {
    FILE* f = fopen(in, "rb");
    if (!f) return 2;
    unsigned n = 0;
    if (fread(&n, 4, 1, f) != 1) return 2;
    std::vector<FracIn> rec(n);
    if (n && fread(rec.data(), sizeof(FracIn), n, f) != n) return 2;
    fclose(f);
    FracIn* din;
    float* dout;
    cudaMalloc(&din, sizeof(FracIn) * (size_t)n + 32);
    cudaMalloc(&dout, 12 * (size_t)n + 16);
    cudaMemcpy(din, rec.data(), sizeof(FracIn) * (size_t)n, cudaMemcpyHostToDevice);
    k_frac<<<(n + 255) / 256, 256>>>(din, dout, n);
    std::vector<float> res(3 * (size_t)n);
    cudaMemcpy(res.data(), dout, 12 * (size_t)n, cudaMemcpyDeviceToHost);
    if (cudaDeviceSynchronize() != cudaSuccess) return 3;
    FILE* g = fopen(out, "wb");
    fwrite(res.data(), 4, res.size(), g);
    fclose(g);
    return 0;
}

static int checks() {
    unsigned long long* bad;
    cudaMalloc(&bad, 8 * sizeof(unsigned long long));
    cudaMemset(bad, 0, 8 * sizeof(unsigned long long));
    k_rcp<<<1024, 256>>>(0, 1ull << 24, bad);
    k_rcp<<<1024, 256>>>(0x4B800000ull, 0x4E000000ull - 0x4B800000ull + 1, bad);
    k_misc<<<1024, 256>>>(1ull << 26, bad + 1);
    k_cvt<<<1024, 256>>>(bad + 6);
    unsigned long long h[8];
    cudaMemcpy(h, bad, sizeof h, cudaMemcpyDeviceToHost);
    const cudaError_t e = cudaDeviceSynchronize();
    printf("rcp_rn %llu\ndraw_index %llu\nphilox_vs_curand %llu\nmod_magic %llu\nisqrt %llu\nweight_f %llu\n"
           "u32_to_f32_rn %llu\n", h[0], h[1], h[2], h[3], h[4], h[5], h[6]);
    cudaFree(bad);
    printf("status %s\n", cudaGetErrorString(e));
    return e != cudaSuccess;
}

static int weights(const char* in, const char* out) {
    FILE* f = fopen(in, "rb");
    if (!f) return 2;
    unsigned n = 0;
    if (fread(&n, 4, 1, f) != 1) return 2;
    std::vector<unsigned> off(n), len(n);
    std::vector<float> s;
    for (unsigned v = 0; v < n; ++v) {
        if (fread(&len[v], 4, 1, f) != 1) return 2;
        off[v] = (unsigned)s.size();
        s.resize(s.size() + len[v]);
        if (len[v] && fread(s.data() + off[v], 4, len[v], f) != len[v]) return 2;
    }
    fclose(f);
    unsigned *doff, *dlen;
    float* ds;
    unsigned long long* dw;
    cudaMalloc(&doff, 4 * (size_t)n + 4);
    cudaMalloc(&dlen, 4 * (size_t)n + 4);
    cudaMalloc(&ds, 4 * s.size() + 4);
    cudaMalloc(&dw, 8 * s.size() + 8);
    cudaMemcpy(doff, off.data(), 4 * (size_t)n, cudaMemcpyHostToDevice);
    cudaMemcpy(dlen, len.data(), 4 * (size_t)n, cudaMemcpyHostToDevice);
    cudaMemcpy(ds, s.data(), 4 * s.size(), cudaMemcpyHostToDevice);
    k_weights<<<(n + 127) / 128, 128>>>(doff, dlen, ds, dw, n);
    std::vector<unsigned long long> w(s.size());
    cudaMemcpy(w.data(), dw, 8 * s.size(), cudaMemcpyDeviceToHost);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return 3;
    FILE* g = fopen(out, "wb");
    fwrite(w.data(), 8, w.size(), g);
    fclose(g);
    return 0;
}

int main(int argc, char** argv) {
    if (argc >= 2 && std::string_view(argv[1]) == "weights" && argc == 4) return weights(argv[2], argv[3]);
    if (argc >= 2 && std::string_view(argv[1]) == "frac" && argc == 4) return frac(argv[2], argv[3]);
    return checks();
}
