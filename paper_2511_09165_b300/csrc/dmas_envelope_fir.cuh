// Envelope low-pass on the CUDA cores, for frames too small to fill the GPU
// with tensor-core tiles (at most 1.5e8 tap products M T L).
//
//   e[d][t] = sum_{x=0..2H} g[x] |y[d][t - H + x]|,  y = 0 outside [0, T)
//
// One CTA per (row, 256 outputs): |y| over the tile and its 2H halo and the
// taps are staged in shared memory; thread j sums its output in tap order with
// FP32 FMAs.  Same definition as the tensor-core kernel, different rounding.
#pragma once

#include "dmas_kernels.cuh"

namespace dmas {

constexpr int kFirTile = 128;  // outputs per CTA (one per thread)
constexpr int kFirMaxH = 511;  // taps up to 1023

struct EnvFirJob {
    const float *y;  // [M][T]
    float *img;      // [M][T]
    int M, T;
    int tt0;         // first time tile (kFirTile outputs) of this job
    int t_tiles;     // time tiles of this job (all: ceil(T / kFirTile))
    unsigned first;  // first CTA of this job in the launch
};

struct EnvFirParams {
    int count;
    int H;
    const float *taps;  // [2H + 1] (device)
    unsigned *err;      // error word (host-checked build)
    EnvFirJob job[kBatchMax];
};

__global__ void __launch_bounds__(kFirTile) envelope_fir_kernel(const __grid_constant__ EnvFirParams p) {
    __shared__ float s_y[kFirTile + 2 * kFirMaxH];
    __shared__ float s_h[2 * kFirMaxH + 1];
    int k = 0;
    while (k + 1 < p.count && p.job[k + 1].first <= blockIdx.x) ++k;
    const EnvFirJob &jb = p.job[k];
    const unsigned local = blockIdx.x - jb.first;
    const int row = (int)(local / (unsigned)jb.t_tiles);
    const int t0 = (jb.tt0 + (int)(local - (unsigned)row * (unsigned)jb.t_tiles)) * kFirTile;
    const int H = p.H, L = 2 * H + 1;
    if (!checked_ok(H >= 0 && H <= kFirMaxH && row < jb.M, p.err)) return;
    const float *yrow = jb.y + (size_t)row * jb.T;
    for (int i = threadIdx.x; i < L; i += kFirTile) s_h[i] = p.taps[i];
    for (int i = threadIdx.x; i < kFirTile + 2 * H; i += kFirTile) {
        const int t = t0 - H + i;
        s_y[i] = (t >= 0 && t < jb.T) ? fabsf(yrow[t]) : 0.0f;
    }
    __syncthreads();
    const int j = threadIdx.x;
    float e = 0.0f;
    for (int x = 0; x < L; ++x) e = fmaf(s_h[x], s_y[j + x], e);
    if (t0 + j < jb.T) jb.img[(size_t)row * jb.T + t0 + j] = e;
}

}  // namespace dmas
