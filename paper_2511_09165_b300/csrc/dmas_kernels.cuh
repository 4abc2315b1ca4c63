// Device code of the DMAS-CF beamformer for sm_103a.
//
//   roots_kernel      per microphone sample: s = sgn(m)|m|^(1/n) (Sec. II-B),
//                     written into a zero-padded channel row so the beamform
//                     kernel never tests bounds (samples outside the frame are
//                     zero).
//   beamform_kernel   one CTA per (group of 8 neighbouring directions, tile of
//                     256 output samples).  The bulk-copy (TMA) engine stages
//                     each microphone's window of roots into shared memory;
//                     each warp owns one direction and each lane 8 samples
//                     (strided by 32, so every gather is one contiguous
//                     128-byte shared-memory row).  Per pixel it accumulates
//                     the power sums P_1..P_n (Eq. power_sum) plus sum x and
//                     sum x^2 in FP32 registers, then applies Newton-Girard
//                     (Eqs. dmas2_impl..dmas5_impl, or the recurrence for
//                     n > 5) and the coherence factor (Eq. cf).
//   (the envelope kernels, |y| then a zero-phase FIR low-pass along t, are in
//   dmas_envelope.cuh)
//
// Every wait on an mbarrier is bounded by wall-clock time (globaltimer); on
// expiry the kernel sets a bit in the plan's error word and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmas {

constexpr int kThreads = 256;      // 8 warps, one direction each
constexpr int kPix = 8;            // scalar kernel: output samples per lane (tile 32 x kPix)
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrBounds = 2u;   // host-checked build: an index left its buffer
constexpr unsigned kWorkSlots = 64;  // beamform work counters per frame (one per launch)
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------------------
// Host-checked build (compiled with DMAS_CHECKED; libdmas_checked.so): the
// kernels test their shared- and global-memory indices before each access.
// A failed test sets kErrBounds in the plan's error word (dmas_plan_check
// reports DMAS_EBOUNDS) and the access is skipped, so the kernel neither
// faults nor traps.  In the normal build every test is a compile-time true and
// costs nothing.
// ---------------------------------------------------------------------------
#ifdef DMAS_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

__device__ __forceinline__ bool checked_ok(bool ok, unsigned *err) {
    if constexpr (kChecked) {
        if (!ok) {
            if (err) atomicOr(err, kErrBounds);
            return false;
        }
    }
    return true;
}

// The CTA's dynamic shared memory (every kernel's extern __shared__ array
// starts there) and its size at launch.
extern __shared__ __align__(128) unsigned char dmas_dyn_smem[];
__device__ __forceinline__ uint32_t dyn_smem_size() {
    uint32_t v;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}
// [a, a + bytes) lies inside the dynamic shared memory (a: shared address)
__device__ __forceinline__ bool smem_in(uint32_t a, uint32_t bytes) {
    const uint32_t base = smem_addr(dmas_dyn_smem);
    return a >= base && a + bytes <= base + dyn_smem_size();
}
__device__ __forceinline__ bool smem_in(const void *p, uint32_t bytes) {
    return smem_in(smem_addr(p), bytes);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Count `bytes` as arrived on the barrier without a copy (the host-checked
// build skips a copy whose range failed its test, and the phase must still
// complete).
__device__ __forceinline__ void mbar_complete_tx_local(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Orders this thread's earlier shared-memory accesses before later async-proxy
// (bulk copy) writes to shared memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier, giving up after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long start = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - start > limit_ns) return false;
    }
    return true;
}

// 1-D bulk copy global -> shared, completion counted in bytes on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// 3-D tensor copy global -> shared, completion counted in bytes on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait that lets the thread sleep in the barrier (up to a few
// microseconds per try) instead of spinning on it, so waiting warps leave
// their issue slots to the warps that compute.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(4000u)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_sleep_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait_sleep(bar, parity)) return true;
    const unsigned long long start = global_ns();
    while (!mbar_try_wait_sleep(bar, parity)) {
        if (global_ns() - start > kWaitLimitNs) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// channel element conversions
// ---------------------------------------------------------------------------
template <typename CH> __device__ __forceinline__ float ld_ch(const CH *p);
template <> __device__ __forceinline__ float ld_ch<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float ld_ch<__half>(const __half *p) {
    return __half2float(*p);
}
template <> __device__ __forceinline__ float ld_ch<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
}
template <typename CH> __device__ __forceinline__ CH to_ch(float v);
template <> __device__ __forceinline__ float to_ch<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_ch<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_ch<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------------------
// K1: signed n-th roots into zero-padded channel rows
// ---------------------------------------------------------------------------
struct RootsParams {
    const float *frame;  // [N][T]
    void *chan;          // [N][row] CH, then (raw != 0) [N][row] the raw samples
    unsigned *work;      // the frame's beamform work counters [kWorkSlots]: set to zero
    int N, T, row, padl, order;
    int raw;             // also write chan1[i][c] = m, the sample the root is taken of
    float inv_order;
};

__device__ __forceinline__ float signed_root(float m, int order, float inv_order) {
    switch (order) {
        case 1: return m;
        case 2: return copysignf(sqrtf(fabsf(m)), m);
        case 3: return cbrtf(m);
        default: return copysignf(powf(fabsf(m), inv_order), m);
    }
}

// Four consecutive channel samples of one row with one vector store (rows
// and the left pad are multiples of 8 samples, so a group never straddles a
// row and starts on a 16-byte boundary for FP32, 8 for 16-bit channels).
template <typename CH> __device__ __forceinline__ void store4(CH *dst, const float (&v)[4]);
template <> __device__ __forceinline__ void store4<float>(float *dst, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
}
template <> __device__ __forceinline__ void store4<__half>(__half *dst, const float (&v)[4]) {
    const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
    *reinterpret_cast<uint2 *>(dst) = make_uint2(*reinterpret_cast<const unsigned *>(&a),
                                                 *reinterpret_cast<const unsigned *>(&b));
}
template <> __device__ __forceinline__ void store4<__nv_bfloat16>(__nv_bfloat16 *dst,
                                                                  const float (&v)[4]) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
    *reinterpret_cast<uint2 *>(dst) = make_uint2(*reinterpret_cast<const unsigned *>(&a),
                                                 *reinterpret_cast<const unsigned *>(&b));
}

// `first` and `stride` count groups of four samples.
template <typename CH>
__device__ __forceinline__ void roots_body(const RootsParams &p, size_t first, size_t stride) {
    const size_t total = (size_t)p.N * (size_t)p.row;
    const size_t groups = total / 4;
    const unsigned row4 = (unsigned)p.row / 4u;
    CH *chan = reinterpret_cast<CH *>(p.chan);
    if (first < kWorkSlots && p.work) p.work[first] = 0u;
    for (size_t gi = first; gi < groups; gi += stride) {
        const size_t i = gi / row4;
        const int c = (int)(gi - i * row4) * 4;
        const float *src = p.frame + i * (size_t)p.T;
        float m[4], r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int t = c + j - p.padl;
            m[j] = (t >= 0 && t < p.T) ? src[t] : 0.0f;
            r[j] = signed_root(m[j], p.order, p.inv_order);
        }
        store4<CH>(chan + gi * 4, r);
        if (p.raw) store4<CH>(chan + total + gi * 4, m);
    }
}

template <typename CH>
__global__ void __launch_bounds__(256) roots_kernel(const __grid_constant__ RootsParams p) {
    roots_body<CH>(p, (size_t)blockIdx.x * blockDim.x + threadIdx.x,
                   (size_t)gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
// Batched launches: up to kBatchMax entries (frames, each with its own plan)
// in one grid.  Entry k owns blocks [start[k], start[k + 1]); the parameters
// of every entry travel in the kernel's parameter space.
// ---------------------------------------------------------------------------
constexpr int kBatchMax = 64;

__device__ __forceinline__ int batch_entry(const unsigned *start, int count, unsigned block) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= block) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct RootsBatch {
    int count;
    unsigned start[kBatchMax + 1];
    RootsParams e[kBatchMax];
};

template <typename CH>
__global__ void __launch_bounds__(256) roots_batch_kernel(const __grid_constant__ RootsBatch b) {
    const int k = batch_entry(b.start, b.count, blockIdx.x);
    const unsigned nb = b.start[k + 1] - b.start[k];
    roots_body<CH>(b.e[k], (size_t)(blockIdx.x - b.start[k]) * blockDim.x + threadIdx.x,
                   (size_t)nb * blockDim.x);
}

// ---------------------------------------------------------------------------
// Newton-Girard: E_n from power sums P[1..n]
// ---------------------------------------------------------------------------
// (the same numbering as dmas_ng_prec: compensated FP32 is zero, the default)
enum { NG_CF32 = 0, NG_F64 = 1, NG_F32 = 2 };

// The paper's pre-expanded equations for n <= 5, the recurrence
// k e_k = sum_{i=1..k} (-1)^(i-1) e_{k-i} P_i above that.
template <int ORDER, typename R>
__device__ __forceinline__ R newton_girard(const R (&P)[ORDER + 1]) {
    if constexpr (ORDER == 1) {
        return P[1];
    } else if constexpr (ORDER == 2) {
        return (R)0.5 * (P[1] * P[1] - P[2]);
    } else if constexpr (ORDER == 3) {
        const R p1 = P[1];
        return (p1 * p1 * p1 + (R)2 * P[3] - (R)3 * p1 * P[2]) * ((R)1 / (R)6);
    } else if constexpr (ORDER == 4) {
        const R p1 = P[1], p2 = P[2], q = p1 * p1;
        return (q * q - (R)6 * P[4] + (R)3 * p2 * p2 - (R)6 * p2 * q + (R)8 * P[3] * p1) *
               ((R)1 / (R)24);
    } else if constexpr (ORDER == 5) {
        const R p1 = P[1], p2 = P[2], p3 = P[3], q = p1 * p1;
        return (q * q * p1 - (R)10 * p2 * q * p1 + (R)15 * p2 * p2 * p1 + (R)20 * p3 * q -
                (R)20 * p3 * p2 - (R)30 * p1 * P[4] + (R)24 * P[5]) *
               ((R)1 / (R)120);
    } else {
        R e[ORDER + 1];
        e[0] = (R)1;
#pragma unroll
        for (int k = 1; k <= ORDER; ++k) {
            R s = (R)0;
#pragma unroll
            for (int i = 1; i <= k; ++i) {
                const R term = e[k - i] * P[i];
                s = (i & 1) ? s + term : s - term;
            }
            e[k] = s / (R)k;
        }
        return e[ORDER];
    }
}

// Double-float ("compensated FP32") numbers: value = hi + lo, |lo| <= ulp(hi)/2.
// Error-free transformations: Knuth's TwoSum and the FMA-based TwoProduct
// (Dekker; Ogita, Rump and Oishi).  The _rn intrinsics keep the compiler from
// fusing or reassociating the steps.
struct dfloat {
    float hi, lo;
};
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
    dfloat s = df_two_sum(x.hi, y.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return df_fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ dfloat df_neg(dfloat x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e));
    return df_fast_two_sum(p, e);
}
// x times a plain float (no low part to carry)
__device__ __forceinline__ dfloat df_mul_f(dfloat x, float y) {
    const float p = __fmul_rn(x.hi, y);
    float e = __fmaf_rn(x.hi, y, -p);
    e = __fmaf_rn(x.lo, y, e);
    return df_fast_two_sum(p, e);
}
// x / k for a small positive integer k, as x times the double-float
// reciprocal of k (hi = 1/k rounded to float, lo = the rest; exact for powers
// of two): relative error near 2^-44, in place of two IEEE divisions per
// step (measured on B300 when this recurrence also served n = 5, interpolated
// 2048 x 16384 frame: beamform 1141 us with the divisions, 946 us as here)
template <int K>
__device__ __forceinline__ dfloat df_div_int(dfloat x) {
    constexpr double r = 1.0 / (double)K;
    constexpr float hi = (float)r;
    constexpr float lo = (float)(r - (double)hi);
    return df_mul(x, dfloat{hi, lo});
}

// e_k = (sum_{i=1..k} (-1)^(i-1) e_{k-i} P_i) / k for k = K..ORDER, in
// double-float (orders above 5)
template <int K, int ORDER>
__device__ __forceinline__ void cf32_step(dfloat (&e)[ORDER + 1], const float (&P)[ORDER + 1]) {
    if constexpr (K <= ORDER) {
        dfloat s = df_mul_f(e[K - 1], P[1]);
#pragma unroll
        for (int i = 2; i <= K; ++i) {
            const dfloat term = df_mul_f(e[K - i], P[i]);
            s = df_add(s, (i & 1) ? term : df_neg(term));
        }
        e[K] = df_div_int<K>(s);
        cf32_step<K + 1, ORDER>(e, P);
    }
}

// ---- compensated Horner form of Eqs. dmas2_impl..dmas5_impl ---------------
// Each pre-expanded equation is a polynomial in P_1 whose coefficients are
// products of the other power sums:
//   2 E_2   = P1^2 - P2
//   6 E_3   = (P1^2 - 3 P2) P1 + 2 P3
//   24 E_4  = ((P1^2 - 6 P2) P1 + 8 P3) P1 + 3 (P2^2 - 2 P4)
//   120 E_5 = (((P1^2 - 10 P2) P1 + 20 P3) P1 + 15 (P2^2 - 2 P4)) P1
//             + 24 P5 - 20 P2 P3
// The coefficients are formed exactly as double-floats (error-free products
// and sums), and the polynomial is evaluated by the compensated Horner scheme
// (Graillat, Langlois and Louvet, 2005): every step's product and sum errors,
// captured by TwoProduct and TwoSum, are summed into a correction polynomial
// evaluated alongside in plain FP32.  The result is as accurate as Horner in
// twice the working precision, rounded to FP32 (error ~ u |E_n| + u^2 times
// the sum of the terms' magnitudes), at about 60 FP32 operations for n = 5
// where the double-float recurrence above takes about 250 (measured on B300,
// 2048 x 16384 interpolated frame: beamform 946 -> 785 us).
//
// TwoSum with the operands ordered by magnitude (Dekker's FastTwoSum after a
// compare and two selects): three FP32 additions on the FMA pipe, the compare
// and selects on the integer/logic pipe, in place of Knuth's six additions.
__device__ __forceinline__ dfloat two_sum_ordered(float a, float b) {
    const float s = __fadd_rn(a, b);
    const bool a_big = fabsf(a) >= fabsf(b);
    const float big = a_big ? a : b, small = a_big ? b : a;
    return {s, __fsub_rn(small, __fsub_rn(s, big))};
}
__device__ __forceinline__ dfloat two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
// k * (hi + lo) for a small integer k: exact product of hi, lo scaled
__device__ __forceinline__ dfloat df_scale(float k, dfloat x) {
    const dfloat p = two_prod(k, x.hi);
    return {p.hi, __fmaf_rn(k, x.lo, p.lo)};
}
// One compensated Horner step: s <- s x + c (c = c.hi + c.lo), the rounding
// errors of the product and the sum, plus c.lo, added into the correction
// polynomial r <- r x + (errors).
__device__ __forceinline__ void comp_horner_step(float &s, float &r, float x, dfloat c) {
    const dfloat p = two_prod(s, x);
    const dfloat t = two_sum_ordered(p.hi, c.hi);
    s = t.hi;
    r = __fmaf_rn(r, x, __fadd_rn(__fadd_rn(p.lo, t.lo), c.lo));
}

// (s + r) / D for the integer denominator D of the pre-expanded equation, as a
// product with the rounded reciprocal (within 1.5 ulp of the quotient; a
// residual correction measured no better in the emulation: worst case over
// random and ill-conditioned sets 19.9 against 18.9 ulp at n = 5)
template <int D>
__device__ __forceinline__ float comp_finish(float s, float r) {
    constexpr float inv = (float)(1.0 / (double)D);
    return __fmul_rn(__fadd_rn(s, r), inv);
}

template <int ORDER>
__device__ __forceinline__ float newton_girard_cf32(const float (&P)[ORDER + 1]) {
    if constexpr (ORDER == 1) {
        return P[1];
    } else if constexpr (ORDER <= 5) {
        const float x = P[1];
        // leading step x * x + c_{n-2}
        const dfloat xx = two_prod(x, x);
        dfloat c;
        if constexpr (ORDER == 2) c = {-P[2], 0.0f};
        else if constexpr (ORDER == 3) c = two_prod(-3.0f, P[2]);
        else if constexpr (ORDER == 4) c = two_prod(-6.0f, P[2]);
        else c = two_prod(-10.0f, P[2]);
        const dfloat t = two_sum_ordered(xx.hi, c.hi);
        float s = t.hi;
        float r = __fadd_rn(__fadd_rn(xx.lo, t.lo), c.lo);
        if constexpr (ORDER == 2) {
            return comp_finish<2>(s, r);
        } else if constexpr (ORDER == 3) {
            comp_horner_step(s, r, x, dfloat{__fmul_rn(2.0f, P[3]), 0.0f});
            return comp_finish<6>(s, r);
        } else {
            // P2^2 - 2 P4 as a double-float
            const dfloat q = two_prod(P[2], P[2]);
            const dfloat d0 = two_sum_ordered(q.hi, __fmul_rn(-2.0f, P[4]));
            const dfloat d = {d0.hi, __fadd_rn(q.lo, d0.lo)};
            if constexpr (ORDER == 4) {
                comp_horner_step(s, r, x, two_prod(8.0f, P[3]));
                comp_horner_step(s, r, x, df_scale(3.0f, d));
                return comp_finish<24>(s, r);
            } else {
                comp_horner_step(s, r, x, two_prod(20.0f, P[3]));
                comp_horner_step(s, r, x, df_scale(15.0f, d));
                // 24 P5 - 20 P2 P3: both products exact, their difference by TwoSum
                const dfloat g24 = two_prod(24.0f, P[5]);
                const dfloat m20 = df_scale(20.0f, two_prod(P[2], P[3]));
                const dfloat g = two_sum_ordered(g24.hi, -m20.hi);
                const float glo = __fadd_rn(__fsub_rn(g24.lo, m20.lo), g.lo);
                comp_horner_step(s, r, x, dfloat{g.hi, glo});
                return comp_finish<120>(s, r);
            }
        }
    } else {
        dfloat e[ORDER + 1];
        e[0] = {1.0f, 0.0f};
        cf32_step<1, ORDER>(e, P);
        return __fadd_rn(e[ORDER].hi, e[ORDER].lo);
    }
}

template <int ORDER, int NGP>
__device__ __forceinline__ float esym_from_power_sums(const float (&P)[ORDER + 1]) {
    if constexpr (NGP == NG_F64) {
        double D[ORDER + 1];
#pragma unroll
        for (int k = 0; k <= ORDER; ++k) D[k] = (double)P[k];
        return (float)newton_girard<ORDER, double>(D);
    } else if constexpr (NGP == NG_CF32) {
        return newton_girard_cf32<ORDER>(P);
    } else {
        return newton_girard<ORDER, float>(P);
    }
}

// ---------------------------------------------------------------------------
// K2: gather + power sums + Newton-Girard + CF
// ---------------------------------------------------------------------------
// CF = A^2 / (N B + eps) with CUDA's fast division (__fdividef: within 2 ulp
// for denominators up to 2^126; N B + eps >= eps > 0).
__device__ __forceinline__ float cf_ratio(float A, float B, float n_mics, float eps) {
    return __fdividef(A * A, fmaf(n_mics, B, eps));
}

struct BeamParams {
    // interpolated-delay pair kernel: 3-D view of the root rows and the raw
    // sample rows, dims (row, N, 2), box (window, 1, 2): one tensor copy
    // stages both windows of a microphone; valid when use_tma != 0
    CUtensorMap tmap;
    const void *chan;    // [N][row] roots, zero padded
    const int *gdir;     // [n_groups * 8] direction index or -1
    const int *gws;      // [n_groups][N] window start relative to t0
    const int *rel;      // [n_groups][N][8] shift relative to window start
    const float *frac;   // [n_groups][N][8] interpolation weight (LINEAR)
    const int *sel;      // LINEAR pair kernel: [n_groups][N][8] byte offset of the staged
                         // sample of pixel t0 (the microphone's block + 4 x rel)
    const float *wf2;    // LINEAR pair kernel: [n_groups][N][8][2] {f, f}, the later sample's weight
    float *y;            // [M][T] E_n (x CF)
    float *cf;           // [M][T] or nullptr
    unsigned *err;       // error word
    int N, T, row, padl, window, mic_chunk, n_groups, n_tiles;
    int M;               // directions (rows of y)
    unsigned item0;      // first work item (time tile x n_groups + group) of this launch
    unsigned n_items;    // work items of this launch
    float n_mics_f, cf_eps;
    int use_cf;
    int pairs;           // pair kernel: pixel pairs per lane (time tile 64 * pairs)
    int stage_bytes;     // persistent pair kernel: bytes of one staging buffer (same for a
                         // whole launch)
    unsigned *work;      // persistent pair kernel: this launch's work counter, zero at launch
    int use_tma;         // interpolated-delay pair kernel: stage by tmap (window <= 256)
};

// Running sums per pixel: P_1..P_n, sum x, sum x^2, where for odd n
// P_n == sum x (s^n = x), so P_n is not kept separately.
template <int ORDER> struct SumLayout {
    static constexpr bool kPnIsA = (ORDER & 1) != 0;
    static constexpr int kNumP = kPnIsA ? ORDER - 1 : ORDER;  // P_1..P_kNumP stored
    static constexpr int kNum = kNumP + 2;                    // + A, B
};

// Accumulate one delayed root s (x rebuilt from it as sgn(s)|s|^n) with weight w.
template <int ORDER, bool WEIGHTED>
__device__ __forceinline__ void accumulate(float (&a)[SumLayout<ORDER>::kNum], float s,
                                           float w) {
    constexpr int NP = SumLayout<ORDER>::kNumP;
    float pw = s;
    if constexpr (NP >= 1) a[0] = WEIGHTED ? fmaf(w, s, a[0]) : a[0] + s;
#pragma unroll
    for (int q = 2; q <= ORDER; ++q) {
        pw *= s;
        if (q <= NP) a[q - 1] = WEIGHTED ? fmaf(w, pw, a[q - 1]) : a[q - 1] + pw;
    }
    const float x = (ORDER & 1) ? pw : copysignf(pw, s);
    a[NP] = WEIGHTED ? fmaf(w, x, a[NP]) : a[NP] + x;
    const float wx = WEIGHTED ? w * x : x;
    a[NP + 1] = fmaf(wx, x, a[NP + 1]);
}

template <int ORDER, bool LINEAR, typename CH, int NGP>
__device__ __forceinline__ void beamform_body(const BeamParams &p, unsigned block) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int NA = SumLayout<ORDER>::kNum;
    constexpr int NP = SumLayout<ORDER>::kNumP;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    const int WS = p.window;
    const int NC = p.mic_chunk;
    CH *win = reinterpret_cast<CH *>(smem + 128);
    const size_t win_bytes = ((size_t)NC * WS * sizeof(CH) + 127) & ~(size_t)127;
    int *s_rel = reinterpret_cast<int *>(smem + 128 + win_bytes);
    float *s_frac = reinterpret_cast<float *>(s_rel + NC * 8);

    const unsigned item = block + p.item0;
    const int tile = (int)(item / (unsigned)p.n_groups);
    const int g = (int)(item - (unsigned)tile * (unsigned)p.n_groups);
    const int t0 = tile * (32 * kPix);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    float acc[kPix][NA];
#pragma unroll
    for (int k = 0; k < kPix; ++k)
#pragma unroll
        for (int j = 0; j < NA; ++j) acc[k][j] = 0.0f;

    const CH *chan = reinterpret_cast<const CH *>(p.chan);
    uint32_t parity = 0;
    for (int c0 = 0; c0 < p.N; c0 += NC) {
        const int nc = min(NC, p.N - c0);
        if (c0 > 0) __syncthreads();  // every warp is done with the previous chunk
        if (warp == 0) {
            const uint32_t row_bytes = (uint32_t)(WS * sizeof(CH));
            const uint32_t tab_bytes = (uint32_t)(nc * 8 * 4);
            if (lane == 0)
                mbar_arrive_expect_tx(bar, nc * row_bytes + tab_bytes * (LINEAR ? 2u : 1u));
            __syncwarp();
            for (int il = lane; il < nc; il += 32) {
                const int i = c0 + il;
                const int x = p.padl + t0 + p.gws[(size_t)g * p.N + i];
                const CH *src = chan + (size_t)i * p.row + x;
                if (checked_ok(x >= 0 && x + WS <= p.row && smem_in(win + (size_t)il * WS, row_bytes),
                               p.err))
                    bulk_g2s(win + (size_t)il * WS, src, row_bytes, bar);
                else
                    mbar_complete_tx_local(bar, row_bytes);
            }
            if (lane == 0) {
                const bool tabs_ok = checked_ok(
                    ((size_t)g * p.N + c0 + nc) <= (size_t)p.n_groups * p.N &&
                        smem_in(s_rel, tab_bytes) && (!LINEAR || smem_in(s_frac, tab_bytes)),
                    p.err);
                if (tabs_ok) {
                    bulk_g2s(s_rel, p.rel + ((size_t)g * p.N + c0) * 8, tab_bytes, bar);
                    if (LINEAR)
                        bulk_g2s(s_frac, p.frac + ((size_t)g * p.N + c0) * 8, tab_bytes, bar);
                } else {
                    mbar_complete_tx_local(bar, tab_bytes * (LINEAR ? 2u : 1u));
                }
            }
        }
        const bool ok = mbar_wait_bounded(bar, parity);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(p.err, kErrTimeout);
                mbar_wait_bounded(bar, parity);  // let copies in flight land
            }
            return;
        }
        parity ^= 1u;

        // microphones unrolled by 2 for nearest-sample delays, not at all for
        // interpolated ones (their 8 pixels already carry two samples each):
        // measured on B300, 2048 x 16384 frame, interpolated FP16 roots n = 5
        // 1187 -> 1024 us and FP32 n = 7 1571 -> 1437 us; nearest FP32 n = 7
        // 727 us by 2 against 745 by 1
        constexpr int kUnroll = LINEAR ? 1 : 2;
#pragma unroll kUnroll
        for (int il = 0; il < nc; ++il) {
            const int off = s_rel[il * 8 + warp];
            const CH *rowp = win + (size_t)il * WS + off + lane;
            if (!checked_ok(off >= 0 && off + 31 + 32 * (kPix - 1) + (LINEAR ? 1 : 0) < WS, p.err))
                continue;
            if constexpr (LINEAR) {
                const float f = s_frac[il * 8 + warp];
                const float w0 = 1.0f - f;
#pragma unroll
                for (int k = 0; k < kPix; ++k) {
                    const float a = ld_ch<CH>(rowp + 32 * k);
                    const float b = ld_ch<CH>(rowp + 32 * k + 1);
                    accumulate<ORDER, true>(acc[k], a, w0);
                    accumulate<ORDER, true>(acc[k], b, f);
                }
            } else {
#pragma unroll
                for (int k = 0; k < kPix; ++k)
                    accumulate<ORDER, false>(acc[k], ld_ch<CH>(rowp + 32 * k), 0.0f);
            }
        }
    }

    const int dir = p.gdir[(size_t)g * 8 + warp];
    if (dir < 0 || !checked_ok(dir < p.M, p.err)) return;
    float *yrow = p.y + (size_t)dir * p.T;
    float *cfrow = p.cf ? p.cf + (size_t)dir * p.T : nullptr;
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
        const int t = t0 + lane + 32 * k;
        if (t >= p.T) continue;
        float P[ORDER + 1];
        P[0] = 0.0f;
#pragma unroll
        for (int q = 1; q <= NP; ++q) P[q] = acc[k][q - 1];
        const float A = acc[k][NP], B = acc[k][NP + 1];
        if constexpr (SumLayout<ORDER>::kPnIsA) P[ORDER] = A;
        const float E = esym_from_power_sums<ORDER, NGP>(P);
        const float cf = cf_ratio(A, B, p.n_mics_f, p.cf_eps);
        yrow[t] = p.use_cf ? E * cf : E;
        if (cfrow) cfrow[t] = cf;
    }
}

// ---------------------------------------------------------------------------
// K2 (FP32 channels up to 5th order): the same gather + power sums on PAIRS of
// output samples per lane with packed f32x2 arithmetic: one FFMA2/FMUL2/FADD2
// does two FP32 operations in one issue slot.  Two kernels:
//  * nearest-sample delays (beamform_x2_run): persistent, lane l and pair k
//    take samples t0 + l + 64k and t0 + l + 32 + 64k, each half loaded by a
//    conflict-free 32-lane shared load;
//  * interpolated delays (beamform_x2_lin_body): one work item per CTA, the
//    same lane layout; the roots kernel also writes the raw samples m as a
//    second zero-padded plane (chan1), and both windows of a microphone are
//    staged, so the loop takes x = m and x^2 from m instead of forming them
//    from the root.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2_t;

// 8-byte shared-memory load into a packed operand (volatile: it must not move
// above the stage's barrier wait)
__device__ __forceinline__ f32x2_t lds_f32x2(uint32_t a) {
    f32x2_t v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ f32x2_t f2_fma(f32x2_t a, f32x2_t b, f32x2_t c) {
    f32x2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2_t f2_mul(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2_t f2_add(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2_t f2_pack(float lo, float hi) {
    f32x2_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void f2_unpack(f32x2_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// magnitude of `mag` with the sign of `sgn`, in both halves
__device__ __forceinline__ f32x2_t f2_copysign(f32x2_t mag, f32x2_t sgn) {
    return (mag & 0x7fffffff7fffffffull) | (sgn & 0x8000000080000000ull);
}

template <int ORDER, bool WEIGHTED>
__device__ __forceinline__ void accumulate2(f32x2_t (&a)[SumLayout<ORDER>::kNum], f32x2_t s,
                                            f32x2_t w) {
    constexpr int NP = SumLayout<ORDER>::kNumP;
    f32x2_t pw = s;
    if constexpr (NP >= 1) a[0] = WEIGHTED ? f2_fma(w, s, a[0]) : f2_add(a[0], s);
#pragma unroll
    for (int q = 2; q <= ORDER; ++q) {
        pw = f2_mul(pw, s);
        if (q <= NP) a[q - 1] = WEIGHTED ? f2_fma(w, pw, a[q - 1]) : f2_add(a[q - 1], pw);
    }
    const f32x2_t x = (ORDER & 1) ? pw : f2_copysign(pw, s);
    a[NP] = WEIGHTED ? f2_fma(w, x, a[NP]) : f2_add(a[NP], x);
    const f32x2_t wx = WEIGHTED ? f2_mul(w, x) : x;
    a[NP + 1] = f2_fma(wx, x, a[NP + 1]);
}

// Nearest-sample delays: one delayed pixel pair into the running sums.  For
// n = 4 and 5 the highest power that only feeds its own sum is folded into
// that sum's FMA instead of being formed first: n = 5 forms r^2, r^3 and
// x = r^3 r^2 and takes P_4 += r^2 r^2 as one FFMA2 (9 packed instructions
// per pixel pair and microphone instead of 10); n = 4 takes P_3 += r^2 r (8
// instead of 9).  The FMA rounds once where the product and the sum rounded
// twice.
template <int ORDER>
__device__ __forceinline__ void accumulate2_plain(f32x2_t (&a)[SumLayout<ORDER>::kNum],
                                                  f32x2_t s) {
    if constexpr (ORDER == 5) {
        const f32x2_t s2 = f2_mul(s, s);
        const f32x2_t s3 = f2_mul(s2, s);
        a[0] = f2_add(a[0], s);
        a[1] = f2_add(a[1], s2);
        a[2] = f2_add(a[2], s3);
        a[3] = f2_fma(s2, s2, a[3]);
        const f32x2_t x = f2_mul(s3, s2);
        a[4] = f2_add(a[4], x);
        a[5] = f2_fma(x, x, a[5]);
    } else if constexpr (ORDER == 4) {
        const f32x2_t s2 = f2_mul(s, s);
        const f32x2_t s4 = f2_mul(s2, s2);
        a[0] = f2_add(a[0], s);
        a[1] = f2_add(a[1], s2);
        a[2] = f2_fma(s2, s, a[2]);
        a[3] = f2_add(a[3], s4);
        const f32x2_t x = f2_copysign(s4, s);
        a[4] = f2_add(a[4], x);
        a[5] = f2_fma(x, x, a[5]);
    } else {
        accumulate2<ORDER, false>(a, s, 0ull);
    }
}

// Interpolated delays without recomputing powers.  Pixel t takes
// (1 - f) p(x) + f p(x + 1) per channel, with x = t + shift; pixel t + 1 takes
// x + 1 and x + 2, so every sample's powers are needed by two pixels.  With
//   S[t] = sum_i p(x_i(t)),   V[t] = sum_i f_i p(x_i(t)),
// both summed over the SAME samples, the interpolated sum is
// S[t] - V[t] + V[t + 1]: each staged sample's powers are formed once, added
// plain and f-weighted, and the loop needs only the weight {f, f}.  (Keeping
// U[t] = sum (1 - f) p instead of S takes the same number of instructions but
// twice the weight registers per microphone in flight: measured on B300 at 80
// registers, the 32-microphone, 2048 x 16384 frame beamforms in 0.78 against
// 0.73 ms.)
//
// The kernel stages two planes per microphone, the root s and the raw sample
// m, so x = m (for odd n, s^n; for even n, |m| = s^n) and x^2 need no powers
// of s: per pixel pair and microphone, n = 5 forms s^2, f s^2 and f m
// (FMUL2) and takes
//   P_1 += s, P_2 += s^2, P_3 += s^2 s, P_4 += s^2 s^2, A += m, B += m m,
//   V_1 += f s, V_2 += f s^2, V_3 += (f s^2) s, V_4 += (f s^2) s^2,
//   V_A += f m, V_B += (f m) m,
// 15 packed instructions against 17 when x and every power of s are formed by
// multiplies.  Each product that the FMA folds rounds once where a multiply
// and an add rounded twice.
template <int ORDER>
__device__ __forceinline__ void accumulate2_svm(f32x2_t (&sa)[SumLayout<ORDER>::kNum],
                                                f32x2_t (&v)[SumLayout<ORDER>::kNum],
                                                f32x2_t s, f32x2_t m, f32x2_t wf) {
    constexpr int NP = SumLayout<ORDER>::kNumP;
    if constexpr (ORDER == 2) {
        const f32x2_t am = m & 0x7fffffff7fffffffull;  // s^2 = |m|
        sa[0] = f2_add(sa[0], s);
        v[0] = f2_fma(wf, s, v[0]);
        sa[1] = f2_add(sa[1], am);
        v[1] = f2_fma(wf, am, v[1]);
    } else if constexpr (ORDER == 3) {
        const f32x2_t u = f2_mul(wf, s);
        sa[0] = f2_add(sa[0], s);
        v[0] = f2_add(v[0], u);
        sa[1] = f2_fma(s, s, sa[1]);
        v[1] = f2_fma(u, s, v[1]);
    } else if constexpr (ORDER == 4) {
        const f32x2_t s2 = f2_mul(s, s);
        const f32x2_t u = f2_mul(wf, s);
        const f32x2_t am = m & 0x7fffffff7fffffffull;  // s^4 = |m|
        sa[0] = f2_add(sa[0], s);
        v[0] = f2_add(v[0], u);
        sa[1] = f2_add(sa[1], s2);
        v[1] = f2_fma(u, s, v[1]);
        sa[2] = f2_fma(s2, s, sa[2]);
        v[2] = f2_fma(u, s2, v[2]);
        sa[3] = f2_add(sa[3], am);
        v[3] = f2_fma(wf, am, v[3]);
    } else if constexpr (ORDER == 5) {
        const f32x2_t s2 = f2_mul(s, s);
        const f32x2_t w2 = f2_mul(wf, s2);
        sa[0] = f2_add(sa[0], s);
        v[0] = f2_fma(wf, s, v[0]);
        sa[1] = f2_add(sa[1], s2);
        v[1] = f2_add(v[1], w2);
        sa[2] = f2_fma(s2, s, sa[2]);
        v[2] = f2_fma(w2, s, v[2]);
        sa[3] = f2_fma(s2, s2, sa[3]);
        v[3] = f2_fma(w2, s2, v[3]);
    }
    const f32x2_t wm = f2_mul(wf, m);
    sa[NP] = f2_add(sa[NP], m);
    v[NP] = f2_add(v[NP], wm);
    sa[NP + 1] = f2_fma(m, m, sa[NP + 1]);
    v[NP + 1] = f2_fma(wm, m, v[NP + 1]);
}

// Order 5, K pixel pairs at once: every product formed before the sums that
// use it, across the pairs, so each product is several instructions ahead
// of its first use.  (Measured on B300, 2048 x 16384 interpolated frame:
// 713.0 -> 710.8 us against one pair after the other, 126 registers.)
template <int K>
__device__ __forceinline__ void accumulate2_svm5_multi(f32x2_t (&sa)[K][SumLayout<5>::kNum],
                                                       f32x2_t (&v)[K][SumLayout<5>::kNum],
                                                       const f32x2_t (&s)[K],
                                                       const f32x2_t (&m)[K], f32x2_t wf) {
    constexpr int NP = SumLayout<5>::kNumP;
    f32x2_t s2[K], w2[K], wm[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s2[k] = f2_mul(s[k], s[k]);
#pragma unroll
    for (int k = 0; k < K; ++k) wm[k] = f2_mul(wf, m[k]);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        sa[k][0] = f2_add(sa[k][0], s[k]);
        v[k][0] = f2_fma(wf, s[k], v[k][0]);
        sa[k][NP] = f2_add(sa[k][NP], m[k]);
        sa[k][NP + 1] = f2_fma(m[k], m[k], sa[k][NP + 1]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) w2[k] = f2_mul(wf, s2[k]);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        sa[k][1] = f2_add(sa[k][1], s2[k]);
        sa[k][2] = f2_fma(s2[k], s[k], sa[k][2]);
        sa[k][3] = f2_fma(s2[k], s2[k], sa[k][3]);
        v[k][NP] = f2_add(v[k][NP], wm[k]);
        v[k][NP + 1] = f2_fma(wm[k], m[k], v[k][NP + 1]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        v[k][1] = f2_add(v[k][1], w2[k]);
        v[k][2] = f2_fma(w2[k], s[k], v[k][2]);
        v[k][3] = f2_fma(w2[k], s2[k], v[k][3]);
    }
}

// Order 3, K pixel pairs at once, ordered as for order 5 above.  (Measured on
// B300, 2048 x 16384 interpolated frame: 0.598 -> 0.594 ms per frame; the same
// ordering at order 4 took 0.811 -> 0.822 ms at 128 registers, so order 4
// keeps the pair-by-pair form.)
template <int K>
__device__ __forceinline__ void accumulate2_svm3_multi(f32x2_t (&sa)[K][SumLayout<3>::kNum],
                                                       f32x2_t (&v)[K][SumLayout<3>::kNum],
                                                       const f32x2_t (&s)[K],
                                                       const f32x2_t (&m)[K], f32x2_t wf) {
    constexpr int NP = SumLayout<3>::kNumP;
    f32x2_t u[K], wm[K];
#pragma unroll
    for (int k = 0; k < K; ++k) u[k] = f2_mul(wf, s[k]);
#pragma unroll
    for (int k = 0; k < K; ++k) wm[k] = f2_mul(wf, m[k]);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        sa[k][0] = f2_add(sa[k][0], s[k]);
        sa[k][1] = f2_fma(s[k], s[k], sa[k][1]);
        sa[k][NP] = f2_add(sa[k][NP], m[k]);
        sa[k][NP + 1] = f2_fma(m[k], m[k], sa[k][NP + 1]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        v[k][0] = f2_add(v[k][0], u[k]);
        v[k][1] = f2_fma(u[k], s[k], v[k][1]);
        v[k][NP] = f2_add(v[k][NP], wm[k]);
        v[k][NP + 1] = f2_fma(wm[k], m[k], v[k][NP + 1]);
    }
}

// The f-weighted part for one sample (root s, raw sample m) in scalar
// arithmetic.
template <int ORDER>
__device__ __forceinline__ void accumulate_vm(float (&v)[SumLayout<ORDER>::kNum], float s,
                                              float m, float w1) {
    constexpr int NP = SumLayout<ORDER>::kNumP;
    float pw = s;
#pragma unroll
    for (int q = 1; q <= NP; ++q) {
        if (q > 1) pw *= s;
        v[q - 1] = fmaf(w1, (q == ORDER) ? fabsf(m) : pw, v[q - 1]);
    }
    const float wm = w1 * m;
    v[NP] += wm;
    v[NP + 1] = fmaf(wm, m, v[NP + 1]);
}

// Interpolated delays, one work item (time tile, direction group) per CTA.
// Lane l and pair k hold the pixels t0 + l + 64k (low half) and t0 + l + 32 +
// 64k (high half), each half one conflict-free 32-lane 4-byte shared load
// from the root window and one from the raw-sample window.
template <int ORDER, int NGP, int PAIRS>
__device__ __forceinline__ void beamform_x2_lin_body(const BeamParams &p, unsigned block) {
    constexpr int kPairs = PAIRS;
    constexpr int kTile = 64 * kPairs;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int NA = SumLayout<ORDER>::kNum;
    constexpr int NP = SumLayout<ORDER>::kNumP;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    const int WS = p.window;
    const int NC = p.mic_chunk;
    // per microphone one 128-byte aligned block: its root window, then its
    // raw-sample window
    const int MBf = ((2 * WS * 4 + 127) & ~127) >> 2;
    float *win = reinterpret_cast<float *>(smem + 128);
    int *s_sel = reinterpret_cast<int *>(smem + 128 + NC * MBf * 4);
    float *s_wf = reinterpret_cast<float *>(s_sel + NC * 8);
    // per-lane partial sums of the sample past the tile: [warp][q][lane]
    float *s_vext = s_wf + NC * 16 + ((threadIdx.x >> 5) * NA * 32 + (threadIdx.x & 31));

    const unsigned item = block + p.item0;
    const int tile = (int)(item / (unsigned)p.n_groups);
    const int g = (int)(item - (unsigned)tile * (unsigned)p.n_groups);
    const int t0 = tile * kTile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // The stage's copies are issued by every warp (warp w: microphones w,
    // w + 8, ..., one per lane), the first chunk's window starts read before
    // the barrier is even initialised, the tables first.  (Measured on B300,
    // 2048 x 16384 frame, compensated Newton-Girard: 785 -> 773 us against
    // all copies issued by warp 0 after the barrier set-up.  A per-CTA
    // %globaltimer probe of that earlier form: 0.2 us to the barrier, 0.5 us
    // for the window starts, 1.4 us issuing the 35 copies, 0.2 us until they
    // landed, 5.1 us of microphone loop, 0.9 us of epilogue.)
    const int *gws = p.gws + (size_t)g * p.N;
    int x_first = 0;
    if (warp + 8 * lane < min(NC, p.N)) x_first = gws[warp + 8 * lane];
    const uint32_t row_bytes = (uint32_t)(WS * 4);
    // Thread 0 sets a chunk's byte count and copies its tables (the first
    // chunk's right after the barrier's initialisation, so one CTA barrier
    // precedes the first window copies).
    auto stage_head = [&](int c0, int nc) {
        const uint32_t tab_bytes = (uint32_t)(nc * 8 * 4);
        mbar_arrive_expect_tx(bar, 2 * nc * row_bytes + 3 * tab_bytes);
        const size_t to = ((size_t)g * p.N + c0) * 8;
        if (checked_ok(((size_t)g * p.N + c0 + nc) <= (size_t)p.n_groups * p.N &&
                           smem_in(s_sel, tab_bytes) && smem_in(s_wf, 2 * tab_bytes),
                       p.err)) {
            bulk_g2s(s_sel, p.sel + to, tab_bytes, bar);
            bulk_g2s(s_wf, p.wf2 + to * 2, 2 * tab_bytes, bar);
        } else {
            mbar_complete_tx_local(bar, 3 * tab_bytes);
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        stage_head(0, min(NC, p.N));
    }
    __syncthreads();  // the barrier and the first byte count are set before any copy lands

    // S (acc) and V (vac) of the lane's pairs (U = S - V); s_vext: V at
    // t0 + 64 PAIRS, the sample past the tile, one microphone per lane
    f32x2_t acc[kPairs][NA], vac[kPairs][NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) {
#pragma unroll
        for (int k = 0; k < kPairs; ++k) acc[k][q] = vac[k][q] = 0ull;
        s_vext[q * 32] = 0.0f;
    }

    const float *chan0 = reinterpret_cast<const float *>(p.chan);
    const float *chan1 = chan0 + (size_t)p.N * p.row;
    uint32_t parity = 0;
    for (int c0 = 0; c0 < p.N; c0 += NC) {
        const int nc = min(NC, p.N - c0);
        if (c0 > 0) {
            __syncthreads();  // every warp is done with the previous chunk
            if (warp + 8 * lane < nc) x_first = gws[c0 + warp + 8 * lane];
            if (threadIdx.x == 0) stage_head(c0, nc);
            __syncthreads();  // the byte count is set before any copy can land
        }
        for (int il = warp + 8 * lane; il < nc; il += kThreads) {
            const int i = c0 + il;
            // a multiple of 8 samples (32 bytes)
            const int x = p.padl + t0 + (il < kThreads ? x_first : gws[i]);
            if (!checked_ok(x >= 0 && x + WS <= p.row && smem_in(win + il * MBf, 2 * row_bytes),
                            p.err)) {
                mbar_complete_tx_local(bar, 2 * row_bytes);
            } else if (p.use_tma) {
                tma_load_3d(win + il * MBf, &p.tmap, x, i, 0, bar);
            } else {
                const size_t o = (size_t)i * p.row + x;
                bulk_g2s(win + il * MBf, chan0 + o, row_bytes, bar);
                bulk_g2s(win + il * MBf + WS, chan1 + o, row_bytes, bar);
            }
        }
        const bool ok = mbar_wait_sleep_bounded(bar, parity);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(p.err, kErrTimeout);
                mbar_wait_bounded(bar, parity);  // let copies in flight land
            }
            return;
        }
        parity ^= 1u;

        // s_sel: byte offset, from the staged windows' base, of the
        // direction's sample for pixel t0 (its microphone's block + 4 x the
        // shift relative to the window start).  Plain loads, so the compiler
        // can move them ahead of the arithmetic of the microphone before.
        const unsigned char *wb = reinterpret_cast<const unsigned char *>(win) + 4 * lane;
        const f32x2_t *wfp = reinterpret_cast<const f32x2_t *>(s_wf) + warp;
#pragma unroll 8
        for (int il = 0; il < nc; ++il) {
            const float *r = reinterpret_cast<const float *>(wb + s_sel[il * 8 + warp]);
            if constexpr (kChecked) {  // the lane's samples inside microphone il's root window
                const unsigned char *blk =
                    reinterpret_cast<const unsigned char *>(win) + il * MBf * 4;
                if (!checked_ok(reinterpret_cast<const unsigned char *>(r) >= blk &&
                                    reinterpret_cast<const unsigned char *>(r + 64 * (kPairs - 1) +
                                                                            33) <= blk + WS * 4 &&
                                    smem_in(wfp + 8 * il, 8),
                                p.err))
                    continue;
            }
            const f32x2_t wf = wfp[8 * il];
            if constexpr (ORDER == 5 || ORDER == 3) {
                f32x2_t sv[kPairs], mv[kPairs];
#pragma unroll
                for (int k = 0; k < kPairs; ++k) {
                    sv[k] = f2_pack(r[64 * k], r[64 * k + 32]);
                    mv[k] = f2_pack(r[WS + 64 * k], r[WS + 64 * k + 32]);
                }
                if constexpr (ORDER == 5) accumulate2_svm5_multi<kPairs>(acc, vac, sv, mv, wf);
                else accumulate2_svm3_multi<kPairs>(acc, vac, sv, mv, wf);
            } else {
#pragma unroll
                for (int k = 0; k < kPairs; ++k)
                    accumulate2_svm<ORDER>(acc[k], vac[k], f2_pack(r[64 * k], r[64 * k + 32]),
                                           f2_pack(r[WS + 64 * k], r[WS + 64 * k + 32]), wf);
            }
        }
        // the sample past the tile lies inside the window (its span covers the
        // last pixel's x + 1)
        if (lane < nc) {
            float ve[NA];
#pragma unroll
            for (int q = 0; q < NA; ++q) ve[q] = s_vext[q * 32];
            for (int il = lane; il < nc; il += 32) {
                const int o = s_sel[il * 8 + warp] + 4 * kTile;  // bytes from win
                if (checked_ok(o >= il * MBf * 4 && o + 4 <= il * MBf * 4 + WS * 4, p.err)) {
                    const float *e = reinterpret_cast<const float *>(
                        reinterpret_cast<const unsigned char *>(win) + o);
                    accumulate_vm<ORDER>(ve, e[0], e[WS], s_wf[(il * 8 + warp) * 2]);
                }
            }
#pragma unroll
            for (int q = 0; q < NA; ++q) s_vext[q * 32] = ve[q];
        }
    }

    const int dir = p.gdir[(size_t)g * 8 + warp];
    if (dir < 0 || !checked_ok(dir < p.M, p.err)) return;
    // sum[t] = S[t] - V[t] + V[t + 1].  Pixel t0 + l + 64k (low half): V[t + 1] is
    // lane l + 1's low half (lane 31: lane 0's high half); t0 + l + 32 + 64k (high
    // half): lane l + 1's high half (lane 31: lane 0's low half of the next pair,
    // or, after the last pair, the sample past the tile summed over the lanes'
    // microphones).
    float vext[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) {
        vext[q] = s_vext[q * 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vext[q] += __shfl_xor_sync(0xffffffffu, vext[q], o);
    }
    float nlo[kPairs][NA], nhi[kPairs][NA];
#pragma unroll
    for (int k = 0; k < kPairs; ++k)
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            float lo, hi;
            f2_unpack(vac[k][q], lo, hi);
            nlo[k][q] = __shfl_sync(0xffffffffu, lo, (lane + 1) & 31);
            nhi[k][q] = __shfl_sync(0xffffffffu, hi, (lane + 1) & 31);
        }
#pragma unroll
    for (int k = 0; k < kPairs; ++k)
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            float slo, shi, vlo, vhi;
            f2_unpack(acc[k][q], slo, shi);
            f2_unpack(vac[k][q], vlo, vhi);
            const float vn_lo = lane < 31 ? nlo[k][q] : nhi[k][q];
            const float vn_hi =
                lane < 31 ? nhi[k][q] : (k + 1 < kPairs ? nlo[(k + 1) % kPairs][q] : vext[q]);
            acc[k][q] = f2_pack((slo - vlo) + vn_lo, (shi - vhi) + vn_hi);
        }
    float *yrow = p.y + (size_t)dir * p.T;
    float *cfrow = p.cf ? p.cf + (size_t)dir * p.T : nullptr;
#pragma unroll
    for (int k = 0; k < kPairs; ++k) {
        float P[2][ORDER + 1], A[2], B[2];
        P[0][0] = P[1][0] = 0.0f;
#pragma unroll
        for (int q = 1; q <= NP; ++q) f2_unpack(acc[k][q - 1], P[0][q], P[1][q]);
        f2_unpack(acc[k][NP], A[0], A[1]);
        f2_unpack(acc[k][NP + 1], B[0], B[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = t0 + lane + 32 * h + 64 * k;
            if (t >= p.T) continue;
            if constexpr (SumLayout<ORDER>::kPnIsA) P[h][ORDER] = A[h];
            const float E = esym_from_power_sums<ORDER, NGP>(P[h]);
            const float cf = cf_ratio(A[h], B[h], p.n_mics_f, p.cf_eps);
            yrow[t] = p.use_cf ? E * cf : E;
            if (cfrow) cfrow[t] = cf;
        }
    }
}

// Nearest-sample delays.  PAIRS pixel pairs per lane: time tile 64 * PAIRS.
// The kernel is persistent: a CTA starts with work item (tile, direction
// group) blockIdx.x and then takes items from a counter shared by the launch,
// at most kPersistItems in all (so its CTAs retire every few tens of
// microseconds and kernels on higher-priority streams get SMs; the grid has
// ceil(items / kPersistItems) CTAs), one stage per (item, microphone chunk),
// through two staging buffers.  Its
// warps run free of each other: a warp waits only for the bulk copy of the
// stage it is about to compute, and the last warp to finish with a buffer
// (counted in shared memory) stages the stage after next into it.  Measured
// on B300 against a static item stride and against CTA-wide barriers per
// stage, both of which left SMs idle at the end or between stages.
//
// Src supplies the items: total(), entry(u) (batch entry of item u), par(e)
// (its parameters) and first(e) (its first item).
// work items per CTA of the persistent kernel (measured on B300, 2048 x 16384
// nearest-sample frame: 2 items 440 us, 4 443 us, 8 447-456 us, 16 468 us)
constexpr int kPersistItems = 2;

struct OneFrame {
    const BeamParams &p;
    __device__ unsigned total() const { return p.n_items; }
    __device__ int entry(unsigned) const { return 0; }
    __device__ const BeamParams &par(int) const { return p; }
    __device__ unsigned first(int) const { return 0; }
};

__device__ __forceinline__ int stage_window_bytes(const BeamParams &p) {
    return (p.mic_chunk * p.window * 4 + 127) & ~127;
}

template <int ORDER, int NGP, int PAIRS, class Src>
__device__ __forceinline__ void beamform_x2_run(const Src &src) {
    constexpr int kPairs = PAIRS;
    constexpr int kTile = 64 * kPairs;
    constexpr int kWarps = kThreads / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int NA = SumLayout<ORDER>::kNum;
    constexpr int NP = SumLayout<ORDER>::kNumP;
    // smem[0, 128): per buffer b: full barrier, finished-warp count, the item
    // and first microphone of the stage it holds, the last stage staged into
    // it; the last staged (item, microphone); abort flag
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int *done_cnt = reinterpret_cast<int *>(smem + 16);
    unsigned *st_item = reinterpret_cast<unsigned *>(smem + 24);
    int *st_c0 = reinterpret_cast<int *>(smem + 32);
    int *last_staged = reinterpret_cast<int *>(smem + 40);
    unsigned *cur_item = reinterpret_cast<unsigned *>(smem + 48);
    int *cur_c0 = reinterpret_cast<int *>(smem + 52);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 56);
    int *n_items = reinterpret_cast<int *>(smem + 60);
    const unsigned total = src.total();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (blockIdx.x >= total) return;
    // every entry of a launch carries the same stage_bytes (the largest) and
    // the launch's work counter (zeroed by the roots kernel before)
    const unsigned stage_bytes = (unsigned)src.par(0).stage_bytes;
    unsigned *work = src.par(0).work;

    // Stage the next stage into buffer bf: the next microphone chunk of the
    // last staged item, else a new item (the CTA's own first, then from the
    // launch's counter); with no work left, complete the buffer's phase
    // empty.  Called by a whole warp, one at a time per CTA.
    auto stage_next = [&](int bf, int stage, bool first) {
        unsigned uu;
        int cc;
        if (first) {
            uu = blockIdx.x;
            cc = 0;
        } else {
            uu = *cur_item;
            cc = *cur_c0;
            const BeamParams &q = src.par(src.entry(uu));
            cc += q.mic_chunk;
            if (cc >= q.N) {
                cc = 0;
                unsigned nxt = total;  // this CTA has had its share
                if (lane == 0 && *n_items < kPersistItems) {
                    nxt = gridDim.x + atomicAdd(work, 1u);
                    ++*n_items;
                }
                uu = __shfl_sync(0xffffffffu, nxt, 0);
            }
        }
        if (uu >= total || *abort_flag) {
            if (lane == 0) {
                st_item[bf] = total;
                mbar_arrive(&bar[bf]);
            }
            return;
        }
        const int e = src.entry(uu);
        const BeamParams &q = src.par(e);
        const unsigned loc = uu - src.first(e) + q.item0;
        const int tile = (int)(loc / (unsigned)q.n_groups);
        const int g = (int)(loc - (unsigned)tile * (unsigned)q.n_groups);
        const int nc = min(q.mic_chunk, q.N - cc);
        unsigned char *buf = smem + 128 + (size_t)bf * stage_bytes;
        float *w = reinterpret_cast<float *>(buf);
        int *rel = reinterpret_cast<int *>(buf + stage_window_bytes(q));
        const uint32_t row_bytes = (uint32_t)(q.window * 4);
        const uint32_t tab_bytes = (uint32_t)(nc * 8 * 4);
        if (lane == 0) {
            *cur_item = uu;
            *cur_c0 = cc;
            st_item[bf] = uu;
            st_c0[bf] = cc;
            last_staged[bf] = stage;
            mbar_arrive_expect_tx(&bar[bf], nc * row_bytes + tab_bytes);
        }
        __syncwarp();
        const float *chan = reinterpret_cast<const float *>(q.chan);
        const int *gws = q.gws + (size_t)g * q.N;
        const int t0 = tile * kTile;
        for (int il = lane; il < nc; il += 32) {
            const int i = cc + il;
            const int x = q.padl + t0 + gws[i];
            if (checked_ok(x >= 0 && x + q.window <= q.row && smem_in(w + il * q.window, row_bytes),
                           q.err))
                bulk_g2s(w + il * q.window, chan + (size_t)i * q.row + x, row_bytes, &bar[bf]);
            else
                mbar_complete_tx_local(&bar[bf], row_bytes);
        }
        if (lane == 0) {
            if (checked_ok(((size_t)g * q.N + cc + nc) <= (size_t)q.n_groups * q.N &&
                               smem_in(rel, tab_bytes),
                           q.err))
                bulk_g2s(rel, q.rel + ((size_t)g * q.N + cc) * 8, tab_bytes, &bar[bf]);
            else
                mbar_complete_tx_local(&bar[bf], tab_bytes);
        }
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        done_cnt[0] = done_cnt[1] = 0;
        last_staged[0] = last_staged[1] = -1;
        *abort_flag = 0;
        *n_items = 1;
        fence_mbar_init();
    }
    __syncthreads();
    if (warp == 0) {  // the first two stages
        stage_next(0, 0, true);
        __syncwarp();
        stage_next(1, 1, false);
    }

    f32x2_t acc[kPairs][NA];

    for (int stage = 0;; ++stage) {
        const int bf = stage & 1;
        const bool ok = __all_sync(0xffffffffu,
                                   mbar_wait_bounded(&bar[bf], (uint32_t)(stage >> 1) & 1u));
        if (!ok) {
            if (lane == 0) {
                atomicOr(src.par(0).err, kErrTimeout);
                *abort_flag = 1;
            }
            break;
        }
        const unsigned u = st_item[bf];
        if (u >= total) break;  // no work left
        const int c0 = st_c0[bf];
        const int e = src.entry(u);
        const BeamParams &p = src.par(e);
        const unsigned loc = u - src.first(e) + p.item0;
        const int tile = (int)(loc / (unsigned)p.n_groups);
        const int g = (int)(loc - (unsigned)tile * (unsigned)p.n_groups);
        const int t0 = tile * kTile;
        const int WS = p.window;
        const int nc = min(p.mic_chunk, p.N - c0);
        const bool last_chunk = c0 + p.mic_chunk >= p.N;
        if (c0 == 0) {
#pragma unroll
            for (int k = 0; k < kPairs; ++k)
#pragma unroll
                for (int q = 0; q < NA; ++q) acc[k][q] = 0ull;
        }

        const unsigned char *buf = smem + 128 + (size_t)bf * stage_bytes;
        const float *w = reinterpret_cast<const float *>(buf);
        const int *s_rel = reinterpret_cast<const int *>(buf + stage_window_bytes(p));
        // unrolled by 4 up to order 3 and by 8 above (measured on B300: two
        // pixel pairs per lane, 2048 x 16384 frame, n = 5: unroll 2 480 us, 4 455
        // us, 8 472 us; four pairs, n = 5: 4 455 us, 8 441 us, and the passive
        // 256-microphone frame 21.99 against 21.22 ms; six pairs, n = 3, passive:
        // 4 14.80 ms, 8 15.11 ms, 2 15.49 ms)
        constexpr int kUnroll = ORDER > 3 ? 8 : 4;
#pragma unroll kUnroll
        for (int il = 0; il < nc; ++il) {
            const int off = s_rel[il * 8 + warp];
            const float *r = w + il * WS + off + lane;
            if (!checked_ok(off >= 0 && off + 31 + 64 * (kPairs - 1) + 32 < WS, p.err)) continue;
#pragma unroll
            for (int k = 0; k < kPairs; ++k)
                accumulate2_plain<ORDER>(acc[k], f2_pack(r[64 * k], r[64 * k + 32]));
        }

        // hand the buffer back (the epilogue below reads registers only); the
        // last warp out stages the stage after next
        __syncwarp();
        int before = 0;
        if (lane == 0) {
            __threadfence_block();
            before = atomicAdd(&done_cnt[bf], 1);
            __threadfence_block();
        }
        __syncwarp();
        before = __shfl_sync(0xffffffffu, before, 0);
        if (before == kWarps - 1) {
            if (lane == 0) done_cnt[bf] = 0;
            __threadfence_block();
            fence_proxy_async_smem();  // the warps' reads before the copy's writes
            stage_next(bf, stage + 2, false);
        }
        const int dir = last_chunk ? p.gdir[(size_t)g * 8 + warp] : -1;
        if (dir >= 0 && checked_ok(dir < p.M, p.err)) {
            float *yrow = p.y + (size_t)dir * p.T;
            float *cfrow = p.cf ? p.cf + (size_t)dir * p.T : nullptr;
#pragma unroll
            for (int k = 0; k < kPairs; ++k) {
                float P[2][ORDER + 1], A[2], B[2];
                P[0][0] = P[1][0] = 0.0f;
#pragma unroll
                for (int q = 1; q <= NP; ++q) f2_unpack(acc[k][q - 1], P[0][q], P[1][q]);
                f2_unpack(acc[k][NP], A[0], A[1]);
                f2_unpack(acc[k][NP + 1], B[0], B[1]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int t = t0 + lane + 32 * h + 64 * k;
                    if (t >= p.T) continue;
                    if constexpr (SumLayout<ORDER>::kPnIsA) P[h][ORDER] = A[h];
                    const float E = esym_from_power_sums<ORDER, NGP>(P[h]);
                    const float cf = cf_ratio(A[h], B[h], p.n_mics_f, p.cf_eps);
                    yrow[t] = p.use_cf ? E * cf : E;
                    if (cfrow) cfrow[t] = cf;
                }
            }
        }
        if (*abort_flag) break;
    }
    // After an abort, let the copies in flight land before the CTA exits.
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        for (int b = 0; b < 2; ++b)
            if (last_staged[b] >= 0) mbar_wait_bounded(&bar[b], (uint32_t)(last_staged[b] >> 1) & 1u);
    }
}

// ---------------------------------------------------------------------------
// __global__ entry points: one frame, or a batch of frames (BeamBatch)
// ---------------------------------------------------------------------------
struct BeamBatch {
    int count;
    unsigned start[kBatchMax + 1];
    BeamParams e[kBatchMax];
};

template <int ORDER, bool LINEAR, typename CH, int NGP>
__global__ void __launch_bounds__(kThreads, 2)
    beamform_kernel(const __grid_constant__ BeamParams p) {
    beamform_body<ORDER, LINEAR, CH, NGP>(p, blockIdx.x);
}

template <int ORDER, bool LINEAR, typename CH, int NGP>
__global__ void __launch_bounds__(kThreads, 2)
    beamform_batch_kernel(const __grid_constant__ BeamBatch b) {
    const int k = batch_entry(b.start, b.count, blockIdx.x);
    beamform_body<ORDER, LINEAR, CH, NGP>(b.e[k], blockIdx.x - b.start[k]);
}

struct ManyFrames {
    const BeamBatch &b;
    __device__ unsigned total() const { return b.start[b.count]; }
    __device__ int entry(unsigned u) const { return batch_entry(b.start, b.count, u); }
    __device__ const BeamParams &par(int e) const { return b.e[e]; }
    __device__ unsigned first(int e) const { return b.start[e]; }
};

// CTAs per SM of the pair kernels (the register budget): nearest-sample
// delays four with two pixel pairs per lane, three with more (four pairs above
// order 3, six up to it); interpolated delays (twice the accumulators, three
// pairs per lane) three up to order 3, two above.
constexpr int pair_ctas_per_sm(bool linear, int order, int pairs) {
    return linear ? (order > 3 ? 2 : 3) : (pairs > 2 ? 3 : 4);
}
template <int ORDER, bool LINEAR, int NGP, int PAIRS>
__global__ void __launch_bounds__(kThreads, pair_ctas_per_sm(LINEAR, ORDER, PAIRS))
    beamform_x2_kernel(const __grid_constant__ BeamParams p) {
    if constexpr (LINEAR) beamform_x2_lin_body<ORDER, NGP, PAIRS>(p, blockIdx.x);
    else beamform_x2_run<ORDER, NGP, PAIRS>(OneFrame{p});
}

template <int ORDER, bool LINEAR, int NGP, int PAIRS>
__global__ void __launch_bounds__(kThreads, pair_ctas_per_sm(LINEAR, ORDER, PAIRS))
    beamform_x2_batch_kernel(const __grid_constant__ BeamBatch b) {
    if constexpr (LINEAR) {
        const int k = batch_entry(b.start, b.count, blockIdx.x);
        beamform_x2_lin_body<ORDER, NGP, PAIRS>(b.e[k], blockIdx.x - b.start[k]);
    } else {
        beamform_x2_run<ORDER, NGP, PAIRS>(ManyFrames{b});
    }
}

}  // namespace dmas
