// Every order at once: DAS and DMAS-2..n, each with and without the
// coherence factor (the algorithms compared in Table I and Fig. 5), from one
// gather of the delayed samples.
//
//   root_planes_kernel   per microphone sample, the planes r_q = sgn(m)|m|^(1/q)
//                        of the upper half of the orders, q = floor(NMAX/2)+1
//                        ..NMAX ([q][mic][row], zero padded like the
//                        single-order root channel); the lower roots follow
//                        from them in registers: r_{q} = sgn(r_{2q}) r_{2q}^2
//                        and m = r_3^3 (or sgn(r_2) r_2^2), so NMAX = 5 stages
//                        3 planes, not 5.
//   beamform_orders_kernel
//                        one CTA per (group of 8 directions, time tile); lane l
//                        of warp w owns direction w and the samples t0 + l and
//                        t0 + l + 32 (+ 64 for the second pair of a 128-sample
//                        tile) as packed f32x2 pixel pairs.  The tensor-copy
//                        engine stages, per microphone, one 3-D box: its window
//                        of every plane, so a chunk of microphones costs one
//                        copy per microphone; two chunks in flight.  Per pixel
//                        the lane keeps, in FP32 registers:
//                          sum x, sum x^2          CF (Eq. cf) and E_1 = DAS
//                          sum |x|                 P_2 of order 2 and P_4 of
//                                                  order 4 (|r_2|^2 = |r_4|^4 = |x|)
//                          P_1..P_{q-1} of r_q     for q = 2..NMAX (Eq. power_sum;
//                                                  P_q of odd q is sum x)
//                        then Newton-Girard per order (Eqs. dmas2_impl..
//                        dmas5_impl) and writes the requested images.
//
// For NMAX = 5 that is 13 running sums and 5 staged roots per sample, against
// 2 + 4 + 5 + 6 + 6 sums and 5 gathers over 5 separate passes.  Nearest-sample
// delays take a 128-sample tile (two pairs per lane), interpolated ones a
// 64-sample tile (one pair: their sums are split in two, S[t] plain and V[t]
// with weight f over the same staged sample, the interpolated sum being
// S[t] - V[t] + V[t + 1], so each staged sample's powers are formed once).
//
// Waits on the stage barriers are bounded as in the single-order kernels.
#pragma once

#include "dmas_launch.cuh"

namespace dmas {

// Orders whose roots are staged: q = kFirst..NMAX.
template <int NMAX> struct OrdersPlanes {
    static constexpr int kFirst = NMAX >= 2 ? NMAX / 2 + 1 : 1;
    static constexpr int kNum = NMAX - kFirst + 1;
};

template <int NMAX> struct OrdersLayout {
    static constexpr int kAbs = NMAX >= 2 ? 1 : 0;  // sum |x| kept
    static constexpr int kNum = 2 + kAbs + NMAX * (NMAX - 1) / 2;
    // index of P_1 of order q; P_2..P_{q-1} follow
    static constexpr int base(int q) { return 2 + kAbs + (q - 2) * (q - 1) / 2; }
};

struct RootPlanesParams {
    const float *frame;  // [N][T]
    float *chan;         // [planes][N][row]: plane j holds r_(kFirst + j)
    size_t plane;        // N * row
    int N, T, row, padl;
};

template <int NMAX>
__global__ void __launch_bounds__(256) root_planes_kernel(const __grid_constant__ RootPlanesParams p) {
    const size_t total = (size_t)p.N * (size_t)p.row;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / (size_t)p.row);
        const int t = (int)(idx - (size_t)i * p.row) - p.padl;
        const float m = (t >= 0 && t < p.T) ? p.frame[(size_t)i * p.T + t] : 0.0f;
        constexpr int F = OrdersPlanes<NMAX>::kFirst;
#pragma unroll
        for (int q = F; q <= NMAX; ++q)
            p.chan[(size_t)(q - F) * p.plane + idx] =
                q == 1 ? m : signed_root(m, q, 1.0f / (float)q);
    }
}

struct OrdersParams {
    // 3-D view of the planes for the tensor-copy engine: dims (row, N,
    // planes), box (window, 1, planes); valid when use_tma != 0 (window <= 256)
    CUtensorMap tmap;
    const float *chan;  // [planes][N][row] staged root planes
    size_t plane;       // elements from one plane to the next (N * row)
    const int *gdir;    // [n_groups * 8] direction index or -1
    const int *gws;     // [n_groups][N] window start relative to t0
    const int *rel;     // [n_groups][N][8] shift relative to the window start
    const float *wf2;   // [n_groups][N][8][2] {f, f} (interpolated delays)
    float *y;           // images [n_images][M][T]
    size_t img;         // elements from one image to the next (M * T)
    float *cf;          // [M][T] or nullptr
    unsigned *err;      // error word
    // image index of order k without (slot[0][k]) and with (slot[1][k]) the
    // coherence factor; -1: not wanted
    int slot[2][kOrdersMaxOrder + 1];
    int N, T, row, padl, window, mic_chunk, n_groups, use_tma;
    int halves;         // interpolated delays: 64-sample pieces per CTA tile (more than 1
                        // only with one microphone chunk, which then takes one staging
                        // buffer)
    float n_mics_f, cf_eps;
};

// Bytes of one microphone's staged block (its plane rows of `window`
// samples), padded to 128 bytes, and of one staging buffer (mic_chunk blocks,
// the chunk's shift table and, interpolated, its weight table).  The host
// computes the same (orders_mic_bytes, orders_stage_bytes).
__device__ __forceinline__ int orders_mic_bytes_dev(int planes, int window) {
    return (planes * window * 4 + 127) & ~127;
}
__device__ __forceinline__ int orders_stage_bytes_dev(int planes, bool lin, int mic_chunk,
                                                      int window) {
    return (mic_chunk * orders_mic_bytes_dev(planes, window) + mic_chunk * 32 +
            (lin ? mic_chunk * 64 : 0) + 127) & ~127;
}

constexpr unsigned long long kAbsMask2 = 0x7fffffff7fffffffull;

// All roots s[q - 1] = r_q, q = 1..NMAX, of a pixel pair from its staged
// ones st[j] = r_(kFirst + j): r_q = sgn(r_2q) r_2q^2, and m = r_3^3 when
// order 3 is staged.
template <int NMAX>
__device__ __forceinline__ void expand_roots(const f32x2_t (&st)[OrdersPlanes<NMAX>::kNum],
                                             f32x2_t (&s)[NMAX]) {
    constexpr int F = OrdersPlanes<NMAX>::kFirst;
#pragma unroll
    for (int q = NMAX; q >= 1; --q) {
        if (q >= F) {
            s[q - 1] = st[q - F];
        } else if (q == 1 && NMAX >= 3) {
            s[0] = f2_mul(f2_mul(s[2], s[2]), s[2]);
        } else {
            s[q - 1] = f2_copysign(f2_mul(s[2 * q - 1], s[2 * q - 1]), s[2 * q - 1]);
        }
    }
}
template <int NMAX>
__device__ __forceinline__ void expand_roots(const float (&st)[OrdersPlanes<NMAX>::kNum],
                                             float (&s)[NMAX]) {
    constexpr int F = OrdersPlanes<NMAX>::kFirst;
#pragma unroll
    for (int q = NMAX; q >= 1; --q) {
        if (q >= F) {
            s[q - 1] = st[q - F];
        } else if (q == 1 && NMAX >= 3) {
            s[0] = s[2] * s[2] * s[2];
        } else {
            s[q - 1] = copysignf(s[2 * q - 1] * s[2 * q - 1], s[2 * q - 1]);
        }
    }
}

// Nearest-sample delays: add one delayed pixel pair (its planes s[0..NMAX-1])
// to the running sums.
template <int NMAX>
__device__ __forceinline__ void accumulate_orders(f32x2_t (&a)[OrdersLayout<NMAX>::kNum],
                                                  const f32x2_t (&s)[NMAX]) {
    const f32x2_t x = s[0];
    a[0] = f2_add(a[0], x);
    a[1] = f2_fma(x, x, a[1]);
    if constexpr (NMAX >= 2) a[2] = f2_add(a[2], x & kAbsMask2);
#pragma unroll
    for (int q = 2; q <= NMAX; ++q) {
        const int b = OrdersLayout<NMAX>::base(q);
        f32x2_t pw = s[q - 1];
        a[b] = f2_add(a[b], pw);
        // r_q^j for j < q - 1 by products; the last power, which feeds only
        // its own sum, folded into that sum's FMA (one instruction fewer per
        // order of three or more)
#pragma unroll
        for (int j = 2; j < q - 1; ++j) {
            pw = f2_mul(pw, s[q - 1]);
            a[b + j - 1] = f2_add(a[b + j - 1], pw);
        }
        if (q >= 3) a[b + q - 2] = f2_fma(pw, s[q - 1], a[b + q - 2]);
    }
}

// Nearest-sample delays, K pixel pairs at once: the same sums as
// accumulate_orders, each step taken for every pair before the next.
template <int NMAX, int K>
__device__ __forceinline__ void accumulate_orders_multi(f32x2_t (&a)[K][OrdersLayout<NMAX>::kNum],
                                                        const f32x2_t (&s)[K][NMAX]) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const f32x2_t x = s[k][0];
        a[k][0] = f2_add(a[k][0], x);
        a[k][1] = f2_fma(x, x, a[k][1]);
        if constexpr (NMAX >= 2) a[k][2] = f2_add(a[k][2], x & kAbsMask2);
    }
#pragma unroll
    for (int q = 2; q <= NMAX; ++q) {
        const int b = OrdersLayout<NMAX>::base(q);
        f32x2_t pw[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            pw[k] = s[k][q - 1];
            a[k][b] = f2_add(a[k][b], pw[k]);
        }
#pragma unroll
        for (int j = 2; j < q - 1; ++j)
#pragma unroll
            for (int k = 0; k < K; ++k) {
                pw[k] = f2_mul(pw[k], s[k][q - 1]);
                a[k][b + j - 1] = f2_add(a[k][b + j - 1], pw[k]);
            }
        if (q >= 3)
#pragma unroll
            for (int k = 0; k < K; ++k) a[k][b + q - 2] = f2_fma(pw[k], s[k][q - 1], a[k][b + q - 2]);
    }
}

// Interpolated delays: every power of the sample goes plain into S and
// f-weighted into V (the (1 - f)-weighted sum is S - V; only the weight {f, f}
// is held per microphone).
template <int NMAX>
__device__ __forceinline__ void accumulate_orders_sv(f32x2_t (&sa)[OrdersLayout<NMAX>::kNum],
                                                     f32x2_t (&v)[OrdersLayout<NMAX>::kNum],
                                                     const f32x2_t (&s)[NMAX], f32x2_t wf) {
    const f32x2_t x = s[0];
    const f32x2_t xx = f2_mul(x, x);
    sa[0] = f2_add(sa[0], x);
    v[0] = f2_fma(wf, x, v[0]);
    sa[1] = f2_add(sa[1], xx);
    v[1] = f2_fma(wf, xx, v[1]);
    if constexpr (NMAX >= 2) {
        const f32x2_t ax = x & kAbsMask2;
        sa[2] = f2_add(sa[2], ax);
        v[2] = f2_fma(wf, ax, v[2]);
    }
#pragma unroll
    for (int q = 2; q <= NMAX; ++q) {
        const int b = OrdersLayout<NMAX>::base(q);
        f32x2_t pw = s[q - 1];
        sa[b] = f2_add(sa[b], pw);
        v[b] = f2_fma(wf, pw, v[b]);
#pragma unroll
        for (int j = 2; j < q; ++j) {
            pw = f2_mul(pw, s[q - 1]);
            sa[b + j - 1] = f2_add(sa[b + j - 1], pw);
            v[b + j - 1] = f2_fma(wf, pw, v[b + j - 1]);
        }
    }
}

// The f-weighted part for one sample in scalar arithmetic (the sample past
// the tile).
template <int NMAX>
__device__ __forceinline__ void accumulate_orders_v(float (&v)[OrdersLayout<NMAX>::kNum],
                                                    const float (&s)[NMAX], float w1) {
    const float x = s[0];
    v[0] = fmaf(w1, x, v[0]);
    v[1] = fmaf(w1, x * x, v[1]);
    if constexpr (NMAX >= 2) v[2] = fmaf(w1, fabsf(x), v[2]);
#pragma unroll
    for (int q = 2; q <= NMAX; ++q) {
        const int b = OrdersLayout<NMAX>::base(q);
        float pw = s[q - 1];
        v[b] = fmaf(w1, pw, v[b]);
#pragma unroll
        for (int j = 2; j < q; ++j) {
            pw *= s[q - 1];
            v[b + j - 1] = fmaf(w1, pw, v[b + j - 1]);
        }
    }
}

// E_K from the running sums of one pixel, written to the images that want it;
// then the next order.
template <int K, int NMAX, int NGP>
__device__ __forceinline__ void emit_orders(const float (&a)[OrdersLayout<NMAX>::kNum], float cf,
                                            const OrdersParams &p, size_t pix) {
    if constexpr (K <= NMAX) {
        const int s0 = p.slot[0][K], s1 = p.slot[1][K];
        if (s0 >= 0 || s1 >= 0) {
            float E;
            if constexpr (K == 1) {
                E = a[0];
            } else {
                float P[K + 1];
                P[0] = 0.0f;
#pragma unroll
                for (int j = 1; j < K; ++j) P[j] = a[OrdersLayout<NMAX>::base(K) + j - 1];
                P[K] = (K & 1) ? a[0] : a[2];
                E = esym_from_power_sums<K, NGP>(P);
            }
            if (s0 >= 0) p.y[(size_t)s0 * p.img + pix] = E;
            if (s1 >= 0) p.y[(size_t)s1 * p.img + pix] = E * cf;
        }
        emit_orders<K + 1, NMAX, NGP>(a, cf, p, pix);
    }
}

// Two CTAs per SM with interpolated delays (twice the running sums), three
// with nearest-sample ones (80 registers; measured on B300, hemisphere frame,
// n = 5: 1.227 ms at two CTAs per SM, 1.145 ms at three).
template <int NMAX, bool LINEAR, int NGP>
__global__ void __launch_bounds__(kThreads, LINEAR ? 2 : 3)
    beamform_orders_kernel(const __grid_constant__ OrdersParams p) {
    constexpr int kPairs = LINEAR ? 1 : 2;
    constexpr int kTile = 64 * kPairs;
    constexpr int NA = OrdersLayout<NMAX>::kNum;
    constexpr int NP = OrdersPlanes<NMAX>::kNum;
    extern __shared__ __align__(128) unsigned char smem[];
    // smem: two stage barriers; two staging buffers (microphone chunks c and
    // c + 1 in flight while chunk c is summed), each [mic][plane][window] (one
    // 128-byte aligned block per microphone), the shift table and
    // (interpolated) the weight table; then the per-lane V of the sample past
    // the tile (interpolated), [warp][q][lane]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    const int WS = p.window;
    const int NC = p.mic_chunk;
    const int MB = orders_mic_bytes_dev(NP, WS) >> 2;  // floats per microphone block
    const int SB = orders_stage_bytes_dev(NP, LINEAR, NC, WS);
    const int n_chunks = (p.N + NC - 1) / NC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // interpolated delays with every microphone in one stage: the CTA's tile is
    // H pieces of kTile samples, summed one after the other from one staged
    // window (fewer CTA starts and less window overhang per output)
    const int H = (LINEAR && p.halves > 1 && n_chunks == 1) ? p.halves : 1;
    float *s_vext = reinterpret_cast<float *>(smem + 128 + (H > 1 ? 1 : 2) * SB) +
                    (warp * NA * 32 + lane);

    const int tile = (int)(blockIdx.x / (unsigned)p.n_groups);
    const int g = (int)(blockIdx.x - (unsigned)tile * (unsigned)p.n_groups);
    const int t0 = tile * kTile * H;

    // Staging microphone chunk ci into buffer ci & 1: thread 0 sets the
    // byte count and copies the tables (stage_head); after a barrier every
    // warp copies its microphones' rows (stage_rows: warp w takes microphones
    // w, w + 8, ..., one per lane), each with its window start `x_lane` read
    // beforehand (for microphone warp + 8 lane of the chunk).  (Measured on
    // B300 for the single-order interpolated-delay kernel: copies issued by
    // every warp instead of warp 0 alone took 12 us off 785.)
    const int *gws = p.gws + (size_t)g * p.N;
    auto stage_head = [&](int ci) {
        unsigned char *bb = smem + 128 + (ci & 1) * SB;
        int *rel = reinterpret_cast<int *>(reinterpret_cast<float *>(bb) + NC * MB);
        float *wf = reinterpret_cast<float *>(rel + NC * 8);
        const int c0 = ci * NC;
        const int nc = min(NC, p.N - c0);
        const uint32_t row_bytes = (uint32_t)(WS * 4);
        const uint32_t tab_bytes = (uint32_t)(nc * 8 * 4);
        mbar_arrive_expect_tx(&bar[ci & 1], (uint32_t)NP * nc * row_bytes + tab_bytes +
                                                (LINEAR ? 2u * tab_bytes : 0u));
        const size_t to = ((size_t)g * p.N + c0) * 8;
        if (checked_ok(((size_t)g * p.N + c0 + nc) <= (size_t)p.n_groups * p.N &&
                           smem_in(rel, tab_bytes) && (!LINEAR || smem_in(wf, 2 * tab_bytes)),
                       p.err)) {
            bulk_g2s(rel, p.rel + to, tab_bytes, &bar[ci & 1]);
            if (LINEAR) bulk_g2s(wf, p.wf2 + to * 2, 2 * tab_bytes, &bar[ci & 1]);
        } else {
            mbar_complete_tx_local(&bar[ci & 1], tab_bytes * (LINEAR ? 3u : 1u));
        }
    };
    auto window_start = [&](int ci) -> int {
        const int il = warp + 8 * lane;
        return il < min(NC, p.N - ci * NC) ? gws[ci * NC + il] : 0;
    };
    auto stage_rows = [&](int ci, int x_lane) {
        float *win = reinterpret_cast<float *>(smem + 128 + (ci & 1) * SB);
        const int c0 = ci * NC;
        const int nc = min(NC, p.N - c0);
        const uint32_t row_bytes = (uint32_t)(WS * 4);
        for (int il = warp + 8 * lane; il < nc; il += kThreads) {
            const int i = c0 + il;
            // a multiple of 8 samples (32 bytes)
            const int x = p.padl + t0 + (il < kThreads ? x_lane : gws[i]);
            if (!checked_ok(x >= 0 && x + WS <= p.row &&
                                smem_in(win + il * MB, (uint32_t)NP * row_bytes),
                            p.err)) {
                mbar_complete_tx_local(&bar[ci & 1], (uint32_t)NP * row_bytes);
            } else if (p.use_tma) {
                tma_load_3d(win + il * MB, &p.tmap, x, i, 0, &bar[ci & 1]);
            } else {
                const float *src = p.chan + (size_t)i * p.row + x;
#pragma unroll
                for (int q = 0; q < NP; ++q)
                    bulk_g2s(win + il * MB + q * WS, src + (size_t)q * p.plane, row_bytes,
                             &bar[ci & 1]);
            }
        }
    };

    const int x0 = window_start(0);
    const int x1 = n_chunks > 1 ? window_start(1) : 0;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        stage_head(0);
        if (n_chunks > 1) stage_head(1);
    }
    __syncthreads();  // the barriers and byte counts are set before any copy lands
    stage_rows(0, x0);
    if (n_chunks > 1) stage_rows(1, x1);

    f32x2_t acc[kPairs][NA];
    f32x2_t vac[LINEAR ? NA : 1];
    for (int h = 0; h < H; ++h) {
    const int th = kTile * h;  // this piece's first sample within the CTA tile
#pragma unroll
    for (int q = 0; q < NA; ++q) {
#pragma unroll
        for (int k = 0; k < kPairs; ++k) acc[k][q] = 0ull;
        if constexpr (LINEAR) {
            vac[q] = 0ull;
            s_vext[q * 32] = 0.0f;
        }
    }

    for (int ci = 0; ci < n_chunks; ++ci) {
        const int b = ci & 1;
        const uint32_t parity = (uint32_t)(ci >> 1) & 1u;
        const bool ok = h > 0 || mbar_wait_sleep_bounded(&bar[b], parity);
        if (h == 0 && __syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(p.err, kErrTimeout);
                // let the copies in flight land: this chunk's and the next one's
                mbar_wait_bounded(&bar[b], parity);
                if (ci + 1 < n_chunks)
                    mbar_wait_bounded(&bar[b ^ 1], (uint32_t)((ci + 1) >> 1) & 1u);
            }
            return;
        }
        const unsigned char *bb = smem + 128 + b * SB;
        const float *win = reinterpret_cast<const float *>(bb);
        const int *s_rel = reinterpret_cast<const int *>(win + NC * MB);
        const float *s_wf = reinterpret_cast<const float *>(s_rel + NC * 8);
        const int nc = min(NC, p.N - ci * NC);

#pragma unroll 8
        for (int il = 0; il < nc; ++il) {
            const int off = s_rel[il * 8 + warp] + th;
            const float *r = win + il * MB + off + lane;
            if (!checked_ok(off >= 0 && off + 31 + 64 * (kPairs - 1) + 32 < WS, p.err)) continue;
            if constexpr (LINEAR) {
                // the weight {f, f} of the direction's entry
                const f32x2_t wf =
                    reinterpret_cast<const f32x2_t *>(s_wf)[il * 8 + warp];
                f32x2_t st[NP], s[NMAX];
#pragma unroll
                for (int q = 0; q < NP; ++q) st[q] = f2_pack(r[q * WS], r[q * WS + 32]);
                expand_roots<NMAX>(st, s);
                accumulate_orders_sv<NMAX>(acc[0], vac, s, wf);
            } else {
                f32x2_t sk[kPairs][NMAX];
#pragma unroll
                for (int k = 0; k < kPairs; ++k) {
                    f32x2_t st[NP];
#pragma unroll
                    for (int q = 0; q < NP; ++q)
                        st[q] = f2_pack(r[q * WS + 64 * k], r[q * WS + 64 * k + 32]);
                    expand_roots<NMAX>(st, sk[k]);
                }
                accumulate_orders_multi<NMAX, kPairs>(acc, sk);
            }
        }
        if constexpr (LINEAR) {
            // the sample past the tile, one microphone per lane
            if (lane < nc) {
                float ve[NA];
#pragma unroll
                for (int q = 0; q < NA; ++q) ve[q] = s_vext[q * 32];
                for (int il = lane; il < nc; il += 32) {
                    if (!checked_ok(s_rel[il * 8 + warp] >= 0 &&
                                        s_rel[il * 8 + warp] + th + kTile < WS,
                                    p.err))
                        continue;
                    const float *r = win + il * MB + s_rel[il * 8 + warp] + th + kTile;
                    float st[NP], sv[NMAX];
#pragma unroll
                    for (int q = 0; q < NP; ++q) st[q] = r[q * WS];
                    expand_roots<NMAX>(st, sv);
                    accumulate_orders_v<NMAX>(ve, sv, s_wf[(il * 8 + warp) * 2]);
                }
#pragma unroll
                for (int q = 0; q < NA; ++q) s_vext[q * 32] = ve[q];
            }
        }
        if (ci + 2 < n_chunks) {
            const int xn = window_start(ci + 2);
            __syncthreads();  // every warp is done with buffer b
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();  // the warps' reads before the copy's writes
                stage_head(ci + 2);
            }
            __syncthreads();  // the byte count is set before any copy lands
            fence_proxy_async_smem();
            stage_rows(ci + 2, xn);
        }
    }

    const int dir = p.gdir[(size_t)g * 8 + warp];
    if (dir < 0 || !checked_ok((size_t)dir * p.T < p.img, p.err)) return;
    if constexpr (LINEAR) {
        // sum[t] = S[t] - V[t] + V[t + 1]: V[t + 1] for lane l's t0 + l is lane l + 1's
        // first half (lane 31: lane 0's second half); for t0 + 32 + l, lane
        // l + 1's second half (lane 31: the sample past the tile, summed over
        // the lanes' microphones).
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            float ve = s_vext[q * 32];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ve += __shfl_xor_sync(0xffffffffu, ve, o);
            float slo, shi, vlo, vhi;
            f2_unpack(acc[0][q], slo, shi);
            f2_unpack(vac[q], vlo, vhi);
            const float nlo = __shfl_sync(0xffffffffu, vlo, (lane + 1) & 31);
            const float nhi = __shfl_sync(0xffffffffu, vhi, (lane + 1) & 31);
            acc[0][q] = f2_pack((slo - vlo) + (lane < 31 ? nlo : nhi),
                                (shi - vhi) + (lane < 31 ? nhi : ve));
        }
    }
#pragma unroll
    for (int k = 0; k < kPairs; ++k) {
        float a[2][NA];
#pragma unroll
        for (int q = 0; q < NA; ++q) f2_unpack(acc[k][q], a[0][q], a[1][q]);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int t = t0 + th + lane + 32 * hh + 64 * k;
            if (t >= p.T) continue;
            const size_t pix = (size_t)dir * p.T + t;
            const float cf = cf_ratio(a[hh][0], a[hh][1], p.n_mics_f, p.cf_eps);
            emit_orders<1, NMAX, NGP>(a[hh], cf, p, pix);
            if (p.cf) p.cf[pix] = cf;
        }
    }
    }  // pieces
}

// Launch of one (NMAX, delay mode, Newton-Girard precision) variant; each
// NMAX is instantiated in its own translation unit (orders_o<NMAX>.cu).
template <int NMAX, bool LINEAR, int NGP>
cudaError_t launch_orders_variant(const OrdersParams &p, unsigned grid, size_t smem,
                                  cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    return launch_kernel(beamform_orders_kernel<NMAX, LINEAR, NGP>, once, err, p, grid, smem, s);
}

template <int NMAX, bool LINEAR>
cudaError_t launch_orders_ng(const OrdersParams &p, int ngp, unsigned grid, size_t smem,
                             cudaStream_t s) {
    switch (ngp) {
        case NG_F64: return launch_orders_variant<NMAX, LINEAR, NG_F64>(p, grid, smem, s);
        case NG_F32: return launch_orders_variant<NMAX, LINEAR, NG_F32>(p, grid, smem, s);
        default: return launch_orders_variant<NMAX, LINEAR, NG_CF32>(p, grid, smem, s);
    }
}

template <int NMAX>
cudaError_t launch_orders(const OrdersParams &p, int linear, int ngp, unsigned grid, size_t smem,
                          cudaStream_t s) {
    if (linear) return launch_orders_ng<NMAX, true>(p, ngp, grid, smem, s);
    return launch_orders_ng<NMAX, false>(p, ngp, grid, smem, s);
}

using OrdersLauncher = cudaError_t (*)(const OrdersParams &, int, int, unsigned, size_t,
                                       cudaStream_t);

}  // namespace dmas
