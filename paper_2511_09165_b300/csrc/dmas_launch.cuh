// Launch helpers for the templated kernels.  Each order's beamform kernels are
// instantiated in their own translation unit (beam_o<n>.cu) so the build runs
// in parallel; dmas_api.cu calls launch_beamform_order<n> through a table.
#pragma once

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "dmas_internal.h"
#include "dmas_kernels.cuh"

namespace dmas {

// A batch travels in the kernel's parameter space (at most 32764 bytes).
static_assert(sizeof(BeamBatch) <= 32764, "BeamBatch exceeds the kernel parameter limit");

// Dynamic shared memory a beamform kernel is allowed to request (the sm_100
// family's per-CTA opt-in maximum, 227 KB).
constexpr int kBeamSmemOptIn = 227 * 1024;

template <typename K, typename P>
cudaError_t launch_kernel(K kern, std::once_flag &once, cudaError_t &attr_err, const P &p,
                          unsigned grid, size_t smem, cudaStream_t s) {
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kBeamSmemOptIn);
    });
    if (attr_err != cudaSuccess) return attr_err;
    kern<<<grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

// Launch of the persistent kernel: `items` work items, at most kPersistItems
// per CTA, and never fewer CTAs than fit on the device at once (occupancy for
// this kernel and shared-memory size, cached per device), so small frames
// still spread over every SM.
template <typename K, typename P>
cudaError_t launch_persistent(K kern, std::once_flag &once, cudaError_t &attr_err, const P &p,
                              unsigned items, size_t smem, cudaStream_t s) {
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kBeamSmemOptIn);
    });
    if (attr_err != cudaSuccess) return attr_err;
    struct Slot { int dev = -1; size_t smem = 0; unsigned ctas = 0; };
    static std::mutex mu;
    static Slot cache[4];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    unsigned resident = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Slot &c : cache)
            if (c.dev == dev && c.smem == smem) resident = c.ctas;
        if (resident == 0) {
            int per_sm = 0, sms = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads,
                                                                   smem)) != cudaSuccess ||
                (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) !=
                    cudaSuccess)
                return e;
            resident = (unsigned)std::max(1, per_sm) * (unsigned)sms;
            std::rotate(cache, cache + 3, cache + 4);
            cache[0] = Slot{dev, smem, resident};
        }
    }
    const unsigned capped = (items + kPersistItems - 1) / kPersistItems;
    kern<<<std::min(items, std::max(capped, resident)), kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

// FP32 channels up to kPairMaxOrder: the pair kernel (kLinPairs pairs per lane
// for interpolated delays; round_pairs(ORDER), or 2 for small frames, and
// persistent for nearest-sample delays, `grid` then counting its work items);
// otherwise the scalar one (the same choice as uses_pair_kernel on the host).
template <int ORDER, bool LINEAR, typename CH, int NGP>
cudaError_t launch_beam_variant(const BeamParams &p, unsigned grid, size_t smem,
                                cudaStream_t s) {
    if constexpr (std::is_same<CH, float>::value && ORDER <= kPairMaxOrder) {
        static std::once_flag once;
        static cudaError_t err = cudaSuccess;
        if constexpr (LINEAR) {
            return launch_kernel(beamform_x2_kernel<ORDER, LINEAR, NGP, kLinPairs>, once, err, p,
                                 grid, smem, s);
        } else if (p.pairs == round_pairs(ORDER)) {
            static std::once_flag once_w;
            static cudaError_t err_w = cudaSuccess;
            return launch_persistent(beamform_x2_kernel<ORDER, LINEAR, NGP, round_pairs(ORDER)>,
                                     once_w, err_w, p, grid, smem, s);
        } else {
            return launch_persistent(beamform_x2_kernel<ORDER, LINEAR, NGP, 2>, once, err, p,
                                     grid, smem, s);
        }
    } else {
        static std::once_flag once;
        static cudaError_t err = cudaSuccess;
        return launch_kernel(beamform_kernel<ORDER, LINEAR, CH, NGP>, once, err, p, grid, smem,
                             s);
    }
}

template <int ORDER, bool LINEAR, typename CH>
cudaError_t launch_beam_ng(const BeamParams &p, int ngp, unsigned grid, size_t smem,
                           cudaStream_t s) {
    switch (ngp) {
        case NG_F64: return launch_beam_variant<ORDER, LINEAR, CH, NG_F64>(p, grid, smem, s);
        case NG_F32: return launch_beam_variant<ORDER, LINEAR, CH, NG_F32>(p, grid, smem, s);
        default: return launch_beam_variant<ORDER, LINEAR, CH, NG_CF32>(p, grid, smem, s);
    }
}

template <int ORDER, bool LINEAR>
cudaError_t launch_beam_ch(const BeamParams &p, int chan, int ngp, unsigned grid, size_t smem,
                           cudaStream_t s) {
    switch (chan) {
        case 1: return launch_beam_ng<ORDER, LINEAR, __half>(p, ngp, grid, smem, s);
        case 2: return launch_beam_ng<ORDER, LINEAR, __nv_bfloat16>(p, ngp, grid, smem, s);
        default: return launch_beam_ng<ORDER, LINEAR, float>(p, ngp, grid, smem, s);
    }
}

template <int ORDER>
cudaError_t launch_beamform_order(const BeamParams &p, int linear, int chan, int ngp,
                                  unsigned grid, size_t smem, cudaStream_t s) {
    if (linear) return launch_beam_ch<ORDER, true>(p, chan, ngp, grid, smem, s);
    return launch_beam_ch<ORDER, false>(p, chan, ngp, grid, smem, s);
}

using BeamLauncher = cudaError_t (*)(const BeamParams &, int, int, int, unsigned, size_t,
                                     cudaStream_t);

// Batched launch of one kernel variant over up to kBatchMax entries.
template <int ORDER, bool LINEAR, typename CH, int NGP>
cudaError_t launch_beam_batch_variant(const BeamBatch &b, unsigned grid, size_t smem,
                                      cudaStream_t s) {
    if constexpr (std::is_same<CH, float>::value && ORDER <= kPairMaxOrder) {
        static std::once_flag once;
        static cudaError_t err = cudaSuccess;
        if constexpr (LINEAR) {
            return launch_kernel(beamform_x2_batch_kernel<ORDER, LINEAR, NGP, kLinPairs>, once,
                                 err, b, grid, smem, s);
        } else if (b.e[0].pairs == round_pairs(ORDER)) {  // a batch's entries share their variant
            static std::once_flag once_w;
            static cudaError_t err_w = cudaSuccess;
            return launch_persistent(
                beamform_x2_batch_kernel<ORDER, LINEAR, NGP, round_pairs(ORDER)>, once_w, err_w,
                b, grid, smem, s);
        } else {
            return launch_persistent(beamform_x2_batch_kernel<ORDER, LINEAR, NGP, 2>, once, err,
                                     b, grid, smem, s);
        }
    } else {
        static std::once_flag once;
        static cudaError_t err = cudaSuccess;
        return launch_kernel(beamform_batch_kernel<ORDER, LINEAR, CH, NGP>, once, err, b, grid,
                             smem, s);
    }
}

template <int ORDER, bool LINEAR, typename CH>
cudaError_t launch_beam_batch_ng(const BeamBatch &b, int ngp, unsigned grid,
                                 size_t smem, cudaStream_t s) {
    switch (ngp) {
        case NG_F64:
            return launch_beam_batch_variant<ORDER, LINEAR, CH, NG_F64>(b, grid, smem, s);
        case NG_F32:
            return launch_beam_batch_variant<ORDER, LINEAR, CH, NG_F32>(b, grid, smem, s);
        default:
            return launch_beam_batch_variant<ORDER, LINEAR, CH, NG_CF32>(b, grid, smem, s);
    }
}

template <int ORDER>
cudaError_t launch_beamform_batch_order(const BeamBatch &b, int linear, int chan, int ngp,
                                        unsigned grid, size_t smem, cudaStream_t s) {
    if (linear) {
        switch (chan) {
            case 1: return launch_beam_batch_ng<ORDER, true, __half>(b, ngp, grid, smem, s);
            case 2:
                return launch_beam_batch_ng<ORDER, true, __nv_bfloat16>(b, ngp, grid, smem, s);
            default: return launch_beam_batch_ng<ORDER, true, float>(b, ngp, grid, smem, s);
        }
    }
    switch (chan) {
        case 1: return launch_beam_batch_ng<ORDER, false, __half>(b, ngp, grid, smem, s);
        case 2:
            return launch_beam_batch_ng<ORDER, false, __nv_bfloat16>(b, ngp, grid, smem, s);
        default: return launch_beam_batch_ng<ORDER, false, float>(b, ngp, grid, smem, s);
    }
}

using BeamBatchLauncher = cudaError_t (*)(const BeamBatch &, int, int, int, unsigned, size_t,
                                          cudaStream_t);

}  // namespace dmas
