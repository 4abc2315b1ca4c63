// Envelope detection of the DMAS-CF path (the paper's third processing step,
// Sec. II): |y| low-pass filtered along t.  Included by dmas_api.cu only.
#pragma once

#include "dmas_kernels.cuh"

namespace dmas {

// ---------------------------------------------------------------------------
// K3: envelope, |y| filtered along t with a zero-phase FIR
//   e[t] = sum_{k=-H..H} h[k] |y[t - k]|,  |y| = 0 outside [0, T).
// One CTA per (direction row, tile of 1024 outputs); each thread computes 4
// consecutive outputs.  The tile's input span, with its halo rounded up to a
// multiple of 4 samples (HA), is staged in shared memory as |y|; a thread then
// reads its inputs as 16-byte vectors (lanes 16 bytes apart: conflict-free)
// and, with H fixed at compile time, every tap is an immediate constant-bank
// operand of its FFMA.  Few registers, so up to 8 CTAs share an SM and hide
// the staging loads of one another.
// ---------------------------------------------------------------------------
constexpr int kEnvThreads = 256;
constexpr int kEnvR = 4;                              // consecutive outputs per thread
constexpr int kEnvTile = kEnvThreads * kEnvR;         // outputs per CTA

struct EnvParams {
    const float *y;   // [M][T]
    float *img;       // [M][T]
    int T, n_tiles, L;
};
struct EnvTaps {
    float h[1023];
};

__host__ __device__ constexpr int env_halo_aligned(int H) { return (H + 3) & ~3; }

// Stage |y| over [t0 - HA, t0 + kEnvTile + HA) into s_abs.
__device__ __forceinline__ void env_stage(const float *__restrict__ y, int T, int t0, int HA,
                                          float *s_abs) {
    const int span = kEnvTile + 2 * HA;
    for (int idx = threadIdx.x; idx < span; idx += kEnvThreads) {
        const int t = t0 - HA + idx;
        s_abs[idx] = (t >= 0 && t < T) ? fabsf(__ldg(y + t)) : 0.0f;
    }
}

template <int HH>
__device__ __forceinline__ void envelope_body(const EnvParams &p, const EnvTaps &taps,
                                              unsigned block) {
    extern __shared__ __align__(16) float s_abs[];
    constexpr int HA = env_halo_aligned(HH);
    constexpr int Q = (kEnvR + HA + HH + 3) / 4;  // float4 loads per thread
    const int rowi = (int)(block / (unsigned)p.n_tiles);
    const int tile = (int)(block - (unsigned)rowi * (unsigned)p.n_tiles);
    const int t0 = tile * kEnvTile;
    env_stage(p.y + (size_t)rowi * p.T, p.T, t0, HA, s_abs);
    __syncthreads();
    // thread i: outputs t0 + 4i + r (r = 0..3); s_abs index of input t - k is
    // 4i + r - k + HA, so the vector loads start at 4i.
    const float4 *src = reinterpret_cast<const float4 *>(s_abs) + threadIdx.x;
    float acc[kEnvR];
#pragma unroll
    for (int r = 0; r < kEnvR; ++r) acc[r] = 0.0f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const float4 v = src[q];
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
#pragma unroll
            for (int r = 0; r < kEnvR; ++r) {
                const int k = r + HA - (4 * q + e);
                if (k >= -HH && k <= HH) acc[r] = fmaf(taps.h[k + HH], vv[e], acc[r]);
            }
        }
    }
    float *img = p.img + (size_t)rowi * p.T;
#pragma unroll
    for (int r = 0; r < kEnvR; ++r) {
        const int t = t0 + kEnvR * threadIdx.x + r;
        if (t < p.T) img[t] = acc[r];
    }
}

// Any FIR length (taps from shared memory, runtime loops).
__device__ __forceinline__ void envelope_generic_body(const EnvParams &p, const EnvTaps &taps,
                                                      unsigned block) {
    extern __shared__ __align__(16) float s_abs[];
    const int H = (p.L - 1) / 2;
    const int HA = env_halo_aligned(H);
    const int rowi = (int)(block / (unsigned)p.n_tiles);
    const int tile = (int)(block - (unsigned)rowi * (unsigned)p.n_tiles);
    const int t0 = tile * kEnvTile;
    float *s_h = s_abs + kEnvTile + 2 * HA;
    for (int k = threadIdx.x; k < p.L; k += kEnvThreads) s_h[k] = taps.h[k];
    env_stage(p.y + (size_t)rowi * p.T, p.T, t0, HA, s_abs);
    __syncthreads();
    float *img = p.img + (size_t)rowi * p.T;
    for (int r = 0; r < kEnvR; ++r) {
        const int o = kEnvR * threadIdx.x + r;  // output offset within the tile
        float acc = 0.0f;
        for (int k = -H; k <= H; ++k) acc = fmaf(s_h[k + H], s_abs[o - k + HA], acc);
        const int t = t0 + o;
        if (t < p.T) img[t] = acc;
    }
}

struct EnvBatch {
    int count;
    unsigned start[kBatchMax + 1];
    EnvParams e[kBatchMax];
};

template <int HH>
__global__ void __launch_bounds__(kEnvThreads)
    envelope_kernel(const __grid_constant__ EnvParams p, const __grid_constant__ EnvTaps taps) {
    envelope_body<HH>(p, taps, blockIdx.x);
}

__global__ void __launch_bounds__(kEnvThreads)
    envelope_generic_kernel(const __grid_constant__ EnvParams p,
                            const __grid_constant__ EnvTaps taps) {
    envelope_generic_body(p, taps, blockIdx.x);
}

// A batch whose entries share one set of taps.
template <int HH>
__global__ void __launch_bounds__(kEnvThreads)
    envelope_batch_kernel(const __grid_constant__ EnvBatch b, const __grid_constant__ EnvTaps taps) {
    const int k = batch_entry(b.start, b.count, blockIdx.x);
    if constexpr (HH >= 0)
        envelope_body<HH>(b.e[k], taps, blockIdx.x - b.start[k]);
    else
        envelope_generic_body(b.e[k], taps, blockIdx.x - b.start[k]);
}

}  // namespace dmas
