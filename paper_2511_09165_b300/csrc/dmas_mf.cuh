// Matched filter (pulse compression) on the CUDA cores:
//
//   mf[i][t] = sum_{k=0}^{L-1} e[k] m[i][t + k],  m = 0 past the frame end
//
// One CTA per (microphone, 2304 outputs): the input window (outputs plus L - 1
// samples ahead) and the emitted signal e are staged in shared memory.  Each
// thread computes kMfR = 9 consecutive outputs from a sliding window of 2 x 9
// samples in registers: per tap one shared load of the next sample (threads
// 9 words apart: an odd stride, so a warp's 32 loads hit 32 different banks),
// one broadcast load of e[k] and 9 FMAs.  Every output sums its taps in order
// k = 0, 1, ..., L - 1, in blocks of 18 taps: each block in FP32, the block
// sums in double-float (Knuth's TwoSum).  A plain FP32 chain over ~1000 taps
// rounds against running sums far larger than its result, and the n-th root
// magnifies what that leaves near zero: with the 2.5 ms chirp at 450 kHz it
// gave eps_peak 5.7e-4 on y at n = 5; the blocked form 8e-7.
#pragma once

#include "dmas_kernels.cuh"

namespace dmas {

constexpr int kMfR = 9;
constexpr int kMfThreads = 256;
constexpr int kMfTile = kMfR * kMfThreads;  // outputs per CTA

// taps rounded up to a multiple of 2 kMfR (the loop takes two blocks a turn)
__host__ __device__ inline int mf_padded(int L) { return (L + 2 * kMfR - 1) / (2 * kMfR) * (2 * kMfR); }
// shared floats a CTA needs: window kMfTile + Lp + 2 kMfR, taps Lp
__host__ __device__ inline int mf_smem_floats(int L) {
    return kMfTile + 2 * mf_padded(L) + 2 * kMfR;
}

struct MfJob {
    const float *in;    // [N][T] microphone samples
    float *out;         // [N][T] matched-filtered samples
    const float *taps;  // [L] emitted signal (device)
    int N, T, L;
    int t_tiles;        // ceil(T / kMfTile)
    unsigned first;     // first CTA of this job in the launch
};

struct MfParams {
    int count;
    MfJob job[kBatchMax];
};

__global__ void __launch_bounds__(kMfThreads) matched_filter_kernel(const __grid_constant__ MfParams p) {
    extern __shared__ float mf_smem[];
    int j = 0;
    while (j + 1 < p.count && p.job[j + 1].first <= blockIdx.x) ++j;
    const MfJob &jb = p.job[j];
    const unsigned local = blockIdx.x - jb.first;
    const int row = (int)(local / (unsigned)jb.t_tiles);
    const int t0 = (int)(local - (unsigned)row * (unsigned)jb.t_tiles) * kMfTile;
    const int Lp = mf_padded(jb.L);
    const int nx = kMfTile + Lp + 2 * kMfR;
    float *s_x = mf_smem;
    float *s_e = mf_smem + nx;
    const float *in = jb.in + (size_t)row * jb.T;
    for (int i = threadIdx.x; i < nx; i += kMfThreads) {
        const int t = t0 + i;
        s_x[i] = t < jb.T ? in[t] : 0.0f;
    }
    for (int i = threadIdx.x; i < Lp; i += kMfThreads) s_e[i] = i < jb.L ? jb.taps[i] : 0.0f;
    __syncthreads();

    const float *w = s_x + kMfR * threadIdx.x;
    float acc[kMfR], hi[kMfR], lo[kMfR], xa[kMfR], xb[kMfR];
#pragma unroll
    for (int r = 0; r < kMfR; ++r) {
        hi[r] = lo[r] = 0.0f;
        xa[r] = w[r];
    }
    for (int kb = 0; kb < Lp; kb += 2 * kMfR) {
#pragma unroll
        for (int r = 0; r < kMfR; ++r) acc[r] = 0.0f;
        // taps kb .. kb + 8: window samples kb .. kb + 17 (xa then xb)
#pragma unroll
        for (int r = 0; r < kMfR; ++r) xb[r] = w[kb + kMfR + r];
#pragma unroll
        for (int q = 0; q < kMfR; ++q) {
            const float e = s_e[kb + q];
#pragma unroll
            for (int r = 0; r < kMfR; ++r)
                acc[r] = fmaf(e, (r + q < kMfR) ? xa[r + q] : xb[r + q - kMfR], acc[r]);
        }
        // taps kb + 9 .. kb + 17: window samples kb + 9 .. kb + 26 (xb then xa)
#pragma unroll
        for (int r = 0; r < kMfR; ++r) xa[r] = w[kb + 2 * kMfR + r];
#pragma unroll
        for (int q = 0; q < kMfR; ++q) {
            const float e = s_e[kb + kMfR + q];
#pragma unroll
            for (int r = 0; r < kMfR; ++r)
                acc[r] = fmaf(e, (r + q < kMfR) ? xb[r + q] : xa[r + q - kMfR], acc[r]);
        }
        // (hi, lo) += block sum, without rounding error (TwoSum)
#pragma unroll
        for (int r = 0; r < kMfR; ++r) {
            const float s = __fadd_rn(hi[r], acc[r]);
            const float bb = __fsub_rn(s, hi[r]);
            const float err = __fadd_rn(__fsub_rn(hi[r], __fsub_rn(s, bb)), __fsub_rn(acc[r], bb));
            hi[r] = s;
            lo[r] = __fadd_rn(lo[r], err);
        }
    }
    float *out = jb.out + (size_t)row * jb.T;
    const int tt = t0 + kMfR * (int)threadIdx.x;
#pragma unroll
    for (int r = 0; r < kMfR; ++r)
        if (tt + r < jb.T) out[tt + r] = __fadd_rn(hi[r], lo[r]);
}

}  // namespace dmas
