// C ABI of the DMAS-CF beamformer (declared in include/dmas.h): plan
// lifecycle, device tables and scratch, and the launch sequence of one frame:
//   roots_kernel -> beamform kernel -> envelope_tc_kernel (tensor cores).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "dmas.h"
#include "dmas_internal.h"
#include "dmas_envelope_fir.cuh"
#include "dmas_mf.cuh"
#include "dmas_envelope_tc.cuh"
#include "dmas_launch.cuh"
#include "dmas_orders.cuh"

namespace dmas {
extern template cudaError_t launch_beamform_order<1>(const BeamParams &, int, int, int, unsigned,
                                                     size_t, cudaStream_t);
extern template cudaError_t launch_beamform_order<2>(const BeamParams &, int, int, int, unsigned,
                                                     size_t, cudaStream_t);
extern template cudaError_t launch_beamform_order<3>(const BeamParams &, int, int, int, unsigned,
                                                     size_t, cudaStream_t);
extern template cudaError_t launch_beamform_order<4>(const BeamParams &, int, int, int, unsigned,
                                                     size_t, cudaStream_t);
extern template cudaError_t launch_beamform_order<5>(const BeamParams &, int, int, int, unsigned,
                                                     size_t, cudaStream_t);
extern template cudaError_t launch_beamform_order<6>(const BeamParams &, int, int, int, unsigned,
                                                     size_t, cudaStream_t);
extern template cudaError_t launch_beamform_order<7>(const BeamParams &, int, int, int, unsigned,
                                                     size_t, cudaStream_t);
extern template cudaError_t launch_beamform_order<8>(const BeamParams &, int, int, int, unsigned,
                                                     size_t, cudaStream_t);

extern template cudaError_t launch_beamform_batch_order<1>(const BeamBatch &, int, int, int,
                                                           unsigned, size_t, cudaStream_t);
extern template cudaError_t launch_beamform_batch_order<2>(const BeamBatch &, int, int, int,
                                                           unsigned, size_t, cudaStream_t);
extern template cudaError_t launch_beamform_batch_order<3>(const BeamBatch &, int, int, int,
                                                           unsigned, size_t, cudaStream_t);
extern template cudaError_t launch_beamform_batch_order<4>(const BeamBatch &, int, int, int,
                                                           unsigned, size_t, cudaStream_t);
extern template cudaError_t launch_beamform_batch_order<5>(const BeamBatch &, int, int, int,
                                                           unsigned, size_t, cudaStream_t);
extern template cudaError_t launch_beamform_batch_order<6>(const BeamBatch &, int, int, int,
                                                           unsigned, size_t, cudaStream_t);
extern template cudaError_t launch_beamform_batch_order<7>(const BeamBatch &, int, int, int,
                                                           unsigned, size_t, cudaStream_t);
extern template cudaError_t launch_beamform_batch_order<8>(const BeamBatch &, int, int, int,
                                                           unsigned, size_t, cudaStream_t);

static const BeamBatchLauncher kBeamBatchLaunchers[9] = {
    nullptr,
    &launch_beamform_batch_order<1>, &launch_beamform_batch_order<2>,
    &launch_beamform_batch_order<3>, &launch_beamform_batch_order<4>,
    &launch_beamform_batch_order<5>, &launch_beamform_batch_order<6>,
    &launch_beamform_batch_order<7>, &launch_beamform_batch_order<8>};

static const BeamLauncher kBeamLaunchers[9] = {
    nullptr,
    &launch_beamform_order<1>, &launch_beamform_order<2>, &launch_beamform_order<3>,
    &launch_beamform_order<4>, &launch_beamform_order<5>, &launch_beamform_order<6>,
    &launch_beamform_order<7>, &launch_beamform_order<8>};

extern template cudaError_t launch_orders<1>(const OrdersParams &, int, int, unsigned, size_t,
                                              cudaStream_t);
extern template cudaError_t launch_orders<2>(const OrdersParams &, int, int, unsigned, size_t,
                                              cudaStream_t);
extern template cudaError_t launch_orders<3>(const OrdersParams &, int, int, unsigned, size_t,
                                              cudaStream_t);
extern template cudaError_t launch_orders<4>(const OrdersParams &, int, int, unsigned, size_t,
                                              cudaStream_t);
extern template cudaError_t launch_orders<5>(const OrdersParams &, int, int, unsigned, size_t,
                                              cudaStream_t);

static const OrdersLauncher kOrdersLaunchers[kOrdersMaxOrder + 1] = {
    nullptr, &launch_orders<1>, &launch_orders<2>, &launch_orders<3>, &launch_orders<4>,
    &launch_orders<5>};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
}  // namespace dmas

using namespace dmas;

// dmas_beamform_host pipelines a large frame (at least 2^22 pixels) in time
// chunks, one per 2^21 pixels, 4 to 16: each chunk's image columns download
// while the next chunk computes (measured on the 2048 x 16384 frame: 2.67 ms
// in 4 chunks, 2.56 in 8, 2.52 in 16, 2.55 in 32, against 2.35 ms for the
// download alone).
constexpr int kHostChunksMin = 4, kHostChunksMax = 16;

struct dmas_plan {
    HostPlan hp;
    int device = 0;
    int *d_gdir = nullptr, *d_gws = nullptr, *d_rel = nullptr, *d_sel = nullptr;
    float *d_frac = nullptr, *d_wf2 = nullptr;
    unsigned *d_err = nullptr;
    void *d_scratch = nullptr;        // root channels (+ y buffer with the envelope)
    size_t chan_bytes = 0, ybuf_bytes = 0, table_bytes = 0;
    float *d_io_frame = nullptr, *d_io_image = nullptr;  // dmas_beamform_host staging
    size_t smem_beam = 0, smem_env = 0;
    float *d_taps_tc = nullptr;       // envelope tap operand, TF32 hi/lo (tc_tap_arrays)
    float *d_taps = nullptr;          // envelope taps [L] (CUDA-core FIR for small frames)
    float *d_mf = nullptr;            // matched filter: the emitted signal [mf_len], or null
    size_t mf_bytes = 0;              // matched-filtered frame in the scratch (0: no filter)
    int num_sms = 148;
    // tensor-core envelope: at most this many tiles per CTA (0: one CTA per SM
    // over all tiles); see dmas_plan_set_envelope_tile_cap
    int env_tile_cap = 0;
    cudaStream_t last_stream = nullptr;
    std::string last_error;
    // stage profiling
    bool profiling = false;
    bool profiled_once = false;
    bool env_ran = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // dmas_beamform_host: the image download stream and one event per chunk
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t chunk_ev[kHostChunksMax] = {};
    // dmas_beamform_orders: root planes, pre-envelope images and the
    // matched-filtered frame; allocated by its first call, grown on demand
    void *d_orders = nullptr;
    size_t orders_bytes = 0;
    // the last tensor maps encoded for this plan (the envelope's view of a y
    // buffer, the interpolated-delay beamform's view of its root rows), reused
    // while the buffer is the same: encoding is host work on every call
    mutable std::mutex map_mu;
    mutable CUtensorMap env_map{}, beam_map{}, env_omap{};
    mutable const void *env_map_ptr = nullptr, *beam_map_ptr = nullptr, *env_omap_ptr = nullptr;
    mutable int env_map_rows = -1, env_omap_rows = -1;
};

namespace {

// ---------------------------------------------------------------------------
// Self-test of the bounded wait: the barrier expects two arrivals and gets one,
// so the phase never completes; the wait must give up and report.
// ---------------------------------------------------------------------------
__global__ void wait_timeout_selftest_kernel(unsigned *err, unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive(&bar);
        if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(err, kErrTimeout);
    }
}


dmas_status cuda_fail(dmas_plan *p, cudaError_t e, const char *what) {
    if (p) p->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return DMAS_ECUDA;
}

void free_plan_memory(dmas_plan *p) {
    cudaFree(p->d_gdir);
    cudaFree(p->d_gws);
    cudaFree(p->d_rel);
    cudaFree(p->d_frac);
    cudaFree(p->d_sel);
    cudaFree(p->d_wf2);
    cudaFree(p->d_err);
    cudaFree(p->d_scratch);
    cudaFree(p->d_io_frame);
    cudaFree(p->d_io_image);
    cudaFree(p->d_taps_tc);
    cudaFree(p->d_taps);
    cudaFree(p->d_mf);
    cudaFree(p->d_orders);
    p->d_orders = nullptr;
    p->orders_bytes = 0;
    p->d_taps_tc = nullptr;
    p->d_taps = nullptr;
    p->d_mf = nullptr;
    for (auto &e : p->ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    for (auto &e : p->chunk_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    p->copy_stream = nullptr;
    p->d_gdir = p->d_gws = p->d_rel = p->d_sel = nullptr;
    p->d_frac = p->d_wf2 = nullptr;
    p->d_err = nullptr;
    p->d_scratch = nullptr;
    p->d_io_frame = p->d_io_image = nullptr;
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
    size_t bytes = std::max<size_t>(src.size() * sizeof(T), 16);
    cudaError_t e = cudaMalloc((void **)dst, bytes);
    if (e != cudaSuccess) return e;
    if (!src.empty())
        e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

size_t beam_smem_bytes(const HostPlan &hp) {
    const size_t eb = chan_elem_bytes(hp.chan_prec);
    const size_t win = ((size_t)hp.mic_chunk * hp.window * eb + 127) & ~(size_t)127;
    const size_t tabs = (size_t)hp.mic_chunk * kGroup * 4 * (hp.delay_mode ? 2 : 1);
    if (uses_raw_rows(hp.chan_prec, hp.order, hp.delay_mode))  // root and raw-sample windows
        return lin_pair_smem_bytes(hp.mic_chunk, hp.window);
    if (uses_pair_kernel(hp.chan_prec, hp.order))  // persistent: two staging buffers
        return 128 + 2 * pair_stage_bytes(hp.mic_chunk, hp.window);
    return 128 + win + tabs;
}

// Shared-memory stages of the tensor-core envelope: as many as fit beside the
// tap operand (kEnvSmemMax, its opt-in below), at most kTcStages.
int env_tc_stages(const HostPlan &hp) {
    if (hp.L == 0) return 0;
    const int H = (hp.L - 1) / 2;
    const int taps = tc_align1k(tc_tap_bytes(H));
    const int room = kEnvSmemMax - 1024 - taps - tc_out_bytes(H);
    return std::min(kTcStages, room / kTcStageBytes);
}

size_t env_smem_bytes(const HostPlan &hp) {
    if (hp.L == 0) return 0;
    // + 1 KB: the kernel aligns its stages to 1024 bytes (the 128-byte swizzle period)
    const int H = (hp.L - 1) / 2;
    return 1024 + (size_t)tc_align1k(tc_tap_bytes(H)) + (size_t)env_tc_stages(hp) * kTcStageBytes +
           (size_t)tc_out_bytes(H);
}

// TF32 rounding (nearest, ties away from zero) of a finite float, as cvt.rna.
float tf32_host(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float y;
    std::memcpy(&y, &u, 4);
    return y;
}

// The tensor-core envelope's tap operand, split into TF32 hi and lo parts.
// g~[w] = h[2H - (w - (HA - H))] (e[t] = sum_k h[k] |y[t - k]|) is the tap
// that multiplies |y[t0 - HA + u]| for output t0 + j at w = u - j.
//  Toeplitz form: T[u'][n] = g~[u' - n] (u' = 0..KB-1, n = 0..31) in the
//  canonical K-major layout, float index (n / 8) 8 KB + (u' / 4) 32 +
//  (n % 8) 4 + u' % 4; hi at 0, lo at 32 KB.
//  Phase form: copy r holds, at index z, the tap for output 4q + r where
//  z = u + 4 q' and q' = Nq - 1 - q:  g~[z - 4 (Nq - 1) - r].
std::vector<float> tc_tap_arrays(const HostPlan &hp) {
    const int H = (hp.L - 1) / 2, HA = tc_halo(H), Z = tc_Z(H);
    if (tc_toeplitz(H)) {
        const int KB = tc_KB(H);
        std::vector<float> out((size_t)64 * KB, 0.0f);
        for (int n = 0; n < 32; ++n) {
            for (int u = 0; u < KB; ++u) {
                const int x = u - n - (HA - H);
                if (x < 0 || x > 2 * H) continue;
                const float gv = hp.taps[2 * H - x];
                const float hi = tf32_host(gv);
                const size_t i = (size_t)(n / 8) * 8 * KB + (size_t)(u / 4) * 32 + (n % 8) * 4 + u % 4;
                out[i] = hi;
                out[(size_t)32 * KB + i] = gv - hi;
            }
        }
        return out;
    }
    std::vector<float> out((size_t)8 * Z, 0.0f);
    for (int r = 0; r < 4; ++r) {
        for (int z = 0; z < Z; ++z) {
            const int w = z - 4 * (kTcNq - 1) - r;
            const int x = w - (HA - H);
            if (x < 0 || x > 2 * H) continue;
            const float gv = hp.taps[2 * H - x];
            const float hi = tf32_host(gv);
            out[(size_t)r * Z + z] = hi;
            out[(size_t)(4 + r) * Z + z] = gv - hi;
        }
    }
    return out;
}

// CTAs of a tensor-core envelope launch over `tiles` tiles: one per SM, each
// looping over its share, or with a cap of `cap` tiles per CTA (cap > 0) at
// least ceil(tiles / cap), so CTAs retire every `cap` tiles and kernels on
// higher-priority streams reach the SMs sooner.
unsigned env_grid(unsigned tiles, int num_sms, int cap) {
    unsigned g = std::min<unsigned>(tiles, (unsigned)num_sms);
    if (cap > 0) g = std::max<unsigned>(g, (tiles + (unsigned)cap - 1) / (unsigned)cap);
    return g;
}

template <bool TOEP>
cudaError_t launch_env_tc_form(const EnvTcParams &ep, unsigned grid, size_t smem,
                               cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] {
        // the kernel also has ~1 KB of static shared memory (barriers, TMEM slot)
        attr = cudaFuncSetAttribute(envelope_tc_kernel<TOEP>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kEnvSmemMax);
    });
    if (attr != cudaSuccess) return attr;
    envelope_tc_kernel<TOEP><<<grid, kTcThreadsWS, smem, s>>>(ep);
    return cudaGetLastError();
}

// the tap operand's form is a function of the filter length alone
cudaError_t launch_env_tc(const EnvTcParams &ep, unsigned grid, size_t smem, cudaStream_t s) {
    return tc_toeplitz(ep.H) ? launch_env_tc_form<true>(ep, grid, smem, s)
                             : launch_env_tc_form<false>(ep, grid, smem, s);
}

// cuTensorMapEncodeTiled, looked up once through the runtime.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
        cudaGetLastError();
    });
    return fn;
}

// `rows` (0: the plan's M) rows of T samples: the every-order pass filters
// several images of one plan in one launch.
EnvTcJob env_job(const dmas_plan *p, const float *ybuf, float *d_image, unsigned first,
                 int rows = 0) {
    if (rows == 0) rows = p->hp.M;
    EnvTcJob j;
    std::memset(&j, 0, sizeof(j));
    j.use_tma = 0;
    if ((p->hp.T & 3) == 0 && ((uintptr_t)ybuf & 15) == 0) {
        std::lock_guard<std::mutex> lock(p->map_mu);
        if (p->env_map_ptr == ybuf && p->env_map_rows == rows) {
            j.tmap = p->env_map;
            j.use_tma = 1;
        } else if (EncodeTiledFn enc = encode_tiled()) {
            cuuint64_t dims[2] = {(cuuint64_t)p->hp.T, (cuuint64_t)rows};
            cuuint64_t strides[1] = {(cuuint64_t)p->hp.T * 4};
            cuuint32_t box[2] = {kTcAtomK, kTcRows};
            cuuint32_t es[2] = {1, 1};
            if (enc(&j.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ybuf, dims, strides, box,
                    es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
                j.use_tma = 1;
                p->env_map = j.tmap;
                p->env_map_ptr = ybuf;
                p->env_map_rows = rows;
            }
        }
    }
    // the image as a tensor-store target (Toeplitz form)
    j.use_tma_store = 0;
    if (tc_toeplitz((p->hp.L - 1) / 2) && (p->hp.T & 3) == 0 && ((uintptr_t)d_image & 15) == 0) {
        std::lock_guard<std::mutex> lock(p->map_mu);
        if (p->env_omap_ptr == d_image && p->env_omap_rows == rows) {
            j.omap = p->env_omap;
            j.use_tma_store = 1;
        } else if (EncodeTiledFn enc = encode_tiled()) {
            cuuint64_t dims[2] = {(cuuint64_t)p->hp.T, (cuuint64_t)rows};
            cuuint64_t strides[1] = {(cuuint64_t)p->hp.T * 4};
            cuuint32_t box[2] = {kTcNq, kTcRows};
            cuuint32_t es[2] = {1, 1};
            if (enc(&j.omap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)d_image, dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
                j.use_tma_store = 1;
                p->env_omap = j.omap;
                p->env_omap_ptr = d_image;
                p->env_omap_rows = rows;
            }
        }
    }
    j.y = ybuf;
    j.img = d_image;
    j.M = rows;
    j.T = p->hp.T;
    j.tt0 = 0;
    j.t_tiles = (p->hp.T + kTcJ - 1) / kTcJ;
    j.first = first;
    return j;
}

unsigned env_tiles(const dmas_plan *p, int rows = 0) {
    if (rows == 0) rows = p->hp.M;
    return (unsigned)(((size_t)rows + kTcRows - 1) / kTcRows *
                      (((size_t)p->hp.T + kTcJ - 1) / kTcJ));
}

// Only tiny frames take the CUDA-core FIR: at most 2e7 tap products (M T L).
// Measured on B300 with the tensor-memory envelope: the 2-D frame, 91 x 4096 x
// 181 = 6.7e7, runs 15.4 us on the tensor cores against 18.4 us on the CUDA
// cores, 150 x 4096 x 181 17.4 against 26.6 us.  A property of the plan, so a
// frame gets the same kernel alone and in a batch.
bool env_on_cuda_cores(const dmas_plan *p) {
    return (double)p->hp.M * (double)p->hp.T * (double)p->hp.L <= 2e7;
}

EnvFirJob fir_job(const dmas_plan *p, const float *ybuf, float *d_image, unsigned first,
                  int rows = 0) {
    EnvFirJob j;
    j.y = ybuf;
    j.img = d_image;
    j.M = rows ? rows : p->hp.M;
    j.T = p->hp.T;
    j.tt0 = 0;
    j.t_tiles = (p->hp.T + kFirTile - 1) / kFirTile;
    j.first = first;
    return j;
}

unsigned fir_ctas(const dmas_plan *p, int rows = 0) {
    return (unsigned)((size_t)(rows ? rows : p->hp.M) * ((p->hp.T + kFirTile - 1) / kFirTile));
}

void mark(dmas_plan *p, int k, cudaStream_t s) {
    if (p->profiling) cudaEventRecord(p->ev[k], s);
}

// Per-frame scratch: root channels, y buffer (with the envelope), the
// matched-filtered frame (with the matched filter), and a 256-byte slot for
// the beamform launches' work counters.
size_t scratch_bytes(const dmas_plan *p) {
    return align256(p->chan_bytes) + align256(p->ybuf_bytes) + align256(p->mf_bytes) + 256;
}
float *mf_buffer(const dmas_plan *p, void *scratch) {
    return (float *)((char *)scratch + align256(p->chan_bytes) + align256(p->ybuf_bytes));
}
unsigned *work_counter(const dmas_plan *p, void *scratch) {
    return (unsigned *)((char *)scratch + align256(p->chan_bytes) + align256(p->ybuf_bytes) +
                        align256(p->mf_bytes));
}

// ---- per-stage launch parameters of one frame ----------------------------
RootsParams roots_params(const dmas_plan *p, const float *d_frame, void *scratch) {
    const HostPlan &hp = p->hp;
    RootsParams rp;
    rp.frame = d_frame;
    rp.chan = scratch;
    rp.work = work_counter(p, scratch);
    rp.raw = uses_raw_rows(hp.chan_prec, hp.order, hp.delay_mode) ? 1 : 0;
    rp.N = hp.N;
    rp.T = hp.T;
    rp.row = hp.row;
    rp.padl = hp.padl;
    rp.order = hp.order;
    rp.inv_order = 1.0f / (float)hp.order;
    return rp;
}

unsigned roots_blocks(const dmas_plan *p) {
    const size_t total = (size_t)p->hp.N * p->hp.row;
    return (unsigned)std::min<size_t>((total + 255) / 256, 148 * 32);
}
// The roots kernels take four samples per thread (rows are multiples of 8).
static_assert(kAlign % 4 == 0, "a roots group of four samples must not straddle a row");
unsigned roots4_blocks(const dmas_plan *p) {
    const size_t groups = (size_t)p->hp.N * p->hp.row / 4;
    return (unsigned)std::min<size_t>((groups + 255) / 256, 148 * 32);
}

// Where y (E_n x CF before the envelope) goes: the image itself without the
// envelope, else d_y or the scratch after the root channels.
float *y_target(const dmas_plan *p, float *d_image, float *d_y, void *scratch) {
    if (p->hp.L == 0) return d_image;
    return d_y ? d_y : (float *)((char *)scratch + align256(p->chan_bytes));
}

BeamParams beam_params(const dmas_plan *p, void *scratch, float *ybuf, float *d_cf) {
    const HostPlan &hp = p->hp;
    BeamParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.use_tma = 0;
    if (uses_raw_rows(hp.chan_prec, hp.order, hp.delay_mode) && hp.window <= kTmaMaxBox) {
        std::lock_guard<std::mutex> lock(p->map_mu);
        if (p->beam_map_ptr == scratch) {
            bp.tmap = p->beam_map;
            bp.use_tma = 1;
        } else if (EncodeTiledFn enc = encode_tiled()) {
            // root rows [N][row], then the raw sample rows: one box per
            // microphone, its window in both
            cuuint64_t dims[3] = {(cuuint64_t)hp.row, (cuuint64_t)hp.N, 2};
            cuuint64_t strides[2] = {(cuuint64_t)hp.row * 4, (cuuint64_t)hp.N * hp.row * 4};
            cuuint32_t box[3] = {(cuuint32_t)hp.window, 1, 2};
            cuuint32_t es[3] = {1, 1, 1};
            if (enc(&bp.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, scratch, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
                bp.use_tma = 1;
                p->beam_map = bp.tmap;
                p->beam_map_ptr = scratch;
            }
        }
    }
    bp.chan = scratch;
    bp.work = work_counter(p, scratch);
    bp.gdir = p->d_gdir;
    bp.gws = p->d_gws;
    bp.rel = p->d_rel;
    bp.frac = p->d_frac;
    bp.sel = p->d_sel;
    bp.wf2 = p->d_wf2;
    bp.y = ybuf;
    bp.cf = d_cf;
    bp.err = p->d_err;
    bp.N = hp.N;
    bp.T = hp.T;
    bp.row = hp.row;
    bp.padl = hp.padl;
    bp.window = hp.window;
    bp.mic_chunk = hp.mic_chunk;
    bp.n_groups = hp.n_groups;
    bp.M = hp.M;
    bp.n_tiles = hp.n_tiles;
    bp.item0 = 0;
    bp.n_items = (unsigned)((size_t)hp.n_groups * hp.n_tiles);
    bp.n_mics_f = (float)hp.N;
    bp.cf_eps = (float)hp.cf_eps;
    bp.use_cf = (hp.flags & DMAS_F_CF) ? 1 : 0;
    bp.pairs = hp.pairs;
    bp.stage_bytes = hp.pairs && !hp.delay_mode ? (int)pair_stage_bytes(hp.mic_chunk, hp.window)
                                                : 0;
    return bp;
}

unsigned beam_blocks(const dmas_plan *p) {
    return (unsigned)((size_t)p->hp.n_groups * p->hp.n_tiles);
}

// Enqueue the whole path for one frame with the given scratch.
MfJob mf_job(const dmas_plan *p, const float *in, void *scratch, unsigned first) {
    MfJob j;
    j.in = in;
    j.out = mf_buffer(p, scratch);
    j.taps = p->d_mf;
    j.N = p->hp.N;
    j.T = p->hp.T;
    j.L = (int)p->hp.mf.size();
    j.t_tiles = (p->hp.T + kMfTile - 1) / kMfTile;
    j.first = first;
    return j;
}

unsigned mf_ctas(const dmas_plan *p) {
    return (unsigned)p->hp.N * (unsigned)((p->hp.T + kMfTile - 1) / kMfTile);
}

cudaError_t launch_mf(const MfParams &mp, unsigned grid, size_t smem, cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(matched_filter_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(float) * mf_smem_floats(kMfMaxLen)));
    });
    if (attr != cudaSuccess) return attr;
    matched_filter_kernel<<<grid, kMfThreads, smem, s>>>(mp);
    return cudaGetLastError();
}

// K0 (with the matched filter) and K1: the roots of the frame, or of its
// matched-filtered copy in the scratch.
dmas_status enqueue_roots(dmas_plan *p, const float *d_frame, void *scratch, cudaStream_t s) {
    if (!p->hp.mf.empty()) {
        MfParams mp{};
        mp.count = 1;
        mp.job[0] = mf_job(p, d_frame, scratch, 0);
        const cudaError_t e =
            launch_mf(mp, mf_ctas(p), sizeof(float) * mf_smem_floats(mp.job[0].L), s);
        if (e != cudaSuccess) return cuda_fail(p, e, "matched_filter_kernel launch");
        d_frame = mf_buffer(p, scratch);
    }
    const RootsParams rp = roots_params(p, d_frame, scratch);
    const unsigned rgrid = roots4_blocks(p);
    switch (p->hp.chan_prec) {
        case DMAS_CH_F16: roots_kernel<__half><<<rgrid, 256, 0, s>>>(rp); break;
        case DMAS_CH_BF16: roots_kernel<__nv_bfloat16><<<rgrid, 256, 0, s>>>(rp); break;
        default: roots_kernel<float><<<rgrid, 256, 0, s>>>(rp); break;
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DMAS_OK : cuda_fail(p, e, "roots_kernel launch");
}

dmas_status enqueue_frame(dmas_plan *p, const float *d_frame, float *d_image, float *d_y,
                          float *d_cf, void *scratch, cudaStream_t s) {
    const HostPlan &hp = p->hp;
    cudaError_t e;
    mark(p, 0, s);
    // K1: roots
    dmas_status st = enqueue_roots(p, d_frame, scratch, s);
    if (st != DMAS_OK) return st;
    mark(p, 1, s);

    // K2: beamform into y (the image itself without the envelope)
    const bool env = hp.L > 0;
    float *ybuf = y_target(p, d_image, d_y, scratch);
    const BeamParams bp = beam_params(p, scratch, ybuf, d_cf);
    e = kBeamLaunchers[hp.order](bp, hp.delay_mode, hp.chan_prec, hp.ng_prec, beam_blocks(p),
                                 p->smem_beam, s);
    if (e != cudaSuccess) return cuda_fail(p, e, "beamform_kernel launch");
    mark(p, 2, s);

    if (!env) {
        if (d_y && d_y != d_image) {
            e = cudaMemcpyAsync(d_y, d_image, sizeof(float) * (size_t)hp.M * hp.T,
                                cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(p, e, "copy of y");
        }
        mark(p, 3, s);
        p->env_ran = false;
        p->profiled_once = p->profiled_once || p->profiling;
        return DMAS_OK;
    }
    // K3: envelope, on the CUDA cores for small frames, else on the tensor cores
    if (env_on_cuda_cores(p)) {
        EnvFirParams fp{};
        fp.count = 1;
        fp.H = (hp.L - 1) / 2;
        fp.taps = p->d_taps;
        fp.err = p->d_err;
        fp.job[0] = fir_job(p, ybuf, d_image, 0);
        envelope_fir_kernel<<<fir_ctas(p), kFirTile, 0, s>>>(fp);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return cuda_fail(p, e, "envelope_fir_kernel launch");
        mark(p, 3, s);
        p->env_ran = true;
        p->profiled_once = p->profiled_once || p->profiling;
        return DMAS_OK;
    }
    EnvTcParams ep{};
    ep.count = 1;
    ep.job[0] = env_job(p, ybuf, d_image, 0);
    ep.total_tiles = env_tiles(p);
    ep.H = (hp.L - 1) / 2;
    ep.n_stages = env_tc_stages(hp);
    ep.taps = p->d_taps_tc;
    ep.err = p->d_err;
    e = launch_env_tc(ep, env_grid(ep.total_tiles, p->num_sms, p->env_tile_cap), p->smem_env, s);
    if (e != cudaSuccess) return cuda_fail(p, e, "envelope_tc_kernel launch");
    mark(p, 3, s);
    p->env_ran = true;
    p->profiled_once = p->profiled_once || p->profiling;
    return DMAS_OK;
}

// The host-buffer path for one frame, in time chunks: chunk c beamforms the
// work items of its time tiles (plus the envelope's halo ahead), filters the
// outputs whose input window is complete, and its image columns download on
// the copy stream while chunk c + 1 computes.  Small frames run in one chunk.
dmas_status enqueue_host_chunks(dmas_plan *p, const float *d_frame, float *d_image,
                                float *h_image, void *scratch, cudaStream_t s) {
    static_assert(kTcJ == kFirTile, "both envelope kernels tile time by the same length");
    const HostPlan &hp = p->hp;
    cudaError_t e;
    mark(p, 0, s);
    dmas_status st = enqueue_roots(p, d_frame, scratch, s);
    if (st != DMAS_OK) return st;
    mark(p, 1, s);
    const bool env = hp.L > 0;
    const int H = env ? (hp.L - 1) / 2 : 0;
    const int bt = hp.tile;                     // beamform time tile
    const int n_et = (hp.T + kTcJ - 1) / kTcJ;  // envelope time tiles
    const int units = env ? n_et : hp.n_tiles;
    const size_t px = (size_t)hp.M * hp.T;
    int K = 1;
    if (px >= ((size_t)1 << 22)) {
        K = (int)std::min<size_t>(kHostChunksMax,
                                  std::max<size_t>(kHostChunksMin, px >> 21));
        K = std::min(K, units / 2);
        if (K < kHostChunksMin) K = 1;
    }
    const unsigned G = (unsigned)hp.n_groups;
    float *ybuf = y_target(p, d_image, nullptr, scratch);
    const bool fir = env && env_on_cuda_cores(p);
    int beam_done = 0;
    for (int c = 0; c < K; ++c) {
        const int u_lo = units * c / K, u_hi = units * (c + 1) / K;
        const int unit = env ? kTcJ : bt;
        const int out_lo = u_lo * unit, out_hi = std::min(hp.T, u_hi * unit);
        const int need = (c == K - 1) ? hp.n_tiles
                                      : std::min(hp.n_tiles, (out_hi + H + bt - 1) / bt);
        if (need > beam_done) {
            BeamParams bp = beam_params(p, scratch, ybuf, nullptr);
            bp.item0 = (unsigned)beam_done * G;
            bp.n_items = (unsigned)(need - beam_done) * G;
            bp.work = work_counter(p, scratch) + c;
            e = kBeamLaunchers[hp.order](bp, hp.delay_mode, hp.chan_prec, hp.ng_prec,
                                         bp.n_items, p->smem_beam, s);
            if (e != cudaSuccess) return cuda_fail(p, e, "beamform_kernel launch");
            beam_done = need;
        }
        if (env && fir) {
            EnvFirParams fp{};
            fp.count = 1;
            fp.H = H;
            fp.taps = p->d_taps;
            fp.err = p->d_err;
            fp.job[0] = fir_job(p, ybuf, d_image, 0);
            fp.job[0].tt0 = u_lo;
            fp.job[0].t_tiles = u_hi - u_lo;
            envelope_fir_kernel<<<(unsigned)hp.M * (unsigned)(u_hi - u_lo), kFirTile, 0, s>>>(fp);
            if ((e = cudaGetLastError()) != cudaSuccess)
                return cuda_fail(p, e, "envelope_fir_kernel launch");
        } else if (env) {
            EnvTcParams ep{};
            ep.count = 1;
            ep.job[0] = env_job(p, ybuf, d_image, 0);
            ep.job[0].tt0 = u_lo;
            ep.job[0].t_tiles = u_hi - u_lo;
            ep.total_tiles = (unsigned)((hp.M + kTcRows - 1) / kTcRows) * (unsigned)(u_hi - u_lo);
            ep.H = H;
            ep.n_stages = env_tc_stages(hp);
            ep.taps = p->d_taps_tc;
            ep.err = p->d_err;
            e = launch_env_tc(ep, env_grid(ep.total_tiles, p->num_sms, p->env_tile_cap),
                              p->smem_env, s);
            if (e != cudaSuccess) return cuda_fail(p, e, "envelope_tc_kernel launch");
        }
        if ((e = cudaEventRecord(p->chunk_ev[c], s)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(p->copy_stream, p->chunk_ev[c], 0)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(h_image + out_lo, sizeof(float) * hp.T, d_image + out_lo,
                                   sizeof(float) * hp.T, sizeof(float) * (out_hi - out_lo),
                                   hp.M, cudaMemcpyDeviceToHost, p->copy_stream)) != cudaSuccess)
            return cuda_fail(p, e, "image download");
    }
    // the stages interleave: the profile shows the whole frame as the beamform
    mark(p, 2, s);
    mark(p, 3, s);
    p->env_ran = false;
    p->profiled_once = p->profiled_once || p->profiling;
    return DMAS_OK;
}

// ---- batches ----------------------------------------------------------------
struct BatchEntry {
    dmas_plan *plan;
    const float *frame;
    float *image;
    void *scratch;
    float *ybuf;
};

// Enqueue a batch: one launch per (stage, kernel variant) for up to kBatchMax
// entries at a time.
dmas_status enqueue_batch(const std::vector<BatchEntry> &v, cudaStream_t s) {
    cudaError_t e;
    // K0: matched filter of the entries that have one
    {
        std::vector<const BatchEntry *> sel;
        for (const auto &x : v)
            if (!x.plan->hp.mf.empty()) sel.push_back(&x);
        for (size_t b0 = 0; b0 < sel.size(); b0 += kBatchMax) {
            MfParams mp{};
            mp.count = (int)std::min<size_t>(kBatchMax, sel.size() - b0);
            unsigned ctas = 0;
            int Lmax = 0;
            for (int k = 0; k < mp.count; ++k) {
                const BatchEntry &x = *sel[b0 + k];
                mp.job[k] = mf_job(x.plan, x.frame, x.scratch, ctas);
                ctas += mf_ctas(x.plan);
                Lmax = std::max(Lmax, mp.job[k].L);
            }
            e = launch_mf(mp, ctas, sizeof(float) * mf_smem_floats(Lmax), s);
            if (e != cudaSuccess) return cuda_fail(sel[b0]->plan, e, "matched filter batch");
        }
    }
    // K1: roots, grouped by channel type
    for (int chan = 0; chan < 3; ++chan) {
        std::vector<const BatchEntry *> sel;
        for (const auto &x : v)
            if (x.plan->hp.chan_prec == chan) sel.push_back(&x);
        for (size_t b0 = 0; b0 < sel.size(); b0 += kBatchMax) {
            RootsBatch rb{};
            rb.count = (int)std::min<size_t>(kBatchMax, sel.size() - b0);
            unsigned blocks = 0;
            for (int k = 0; k < rb.count; ++k) {
                const BatchEntry &x = *sel[b0 + k];
                rb.start[k] = blocks;
                rb.e[k] = roots_params(x.plan,
                                       x.plan->hp.mf.empty() ? x.frame : mf_buffer(x.plan, x.scratch),
                                       x.scratch);
                blocks += roots4_blocks(x.plan);
            }
            rb.start[rb.count] = blocks;
            if (chan == DMAS_CH_F16) roots_batch_kernel<__half><<<blocks, 256, 0, s>>>(rb);
            else if (chan == DMAS_CH_BF16) roots_batch_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(rb);
            else roots_batch_kernel<float><<<blocks, 256, 0, s>>>(rb);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(sel[b0]->plan, e, "roots batch");
        }
    }
    // K2: beamform, grouped by kernel variant
    std::vector<bool> done(v.size(), false);
    for (size_t i = 0; i < v.size(); ++i) {
        if (done[i]) continue;
        const HostPlan &a = v[i].plan->hp;
        std::vector<size_t> cls;
        for (size_t j = i; j < v.size(); ++j) {
            const HostPlan &b = v[j].plan->hp;
            if (!done[j] && b.order == a.order && b.delay_mode == a.delay_mode &&
                b.chan_prec == a.chan_prec && b.ng_prec == a.ng_prec && b.pairs == a.pairs) {
                cls.push_back(j);
                done[j] = true;
            }
        }
        for (size_t b0 = 0; b0 < cls.size(); b0 += kBatchMax) {
            BeamBatch bb{};
            bb.count = (int)std::min<size_t>(kBatchMax, cls.size() - b0);
            unsigned blocks = 0;
            size_t smem = 0;
            for (int k = 0; k < bb.count; ++k) {
                const BatchEntry &x = v[cls[b0 + k]];
                bb.start[k] = blocks;
                bb.e[k] = beam_params(x.plan, x.scratch, x.ybuf, nullptr);
                blocks += beam_blocks(x.plan);
                smem = std::max(smem, x.plan->smem_beam);
            }
            bb.start[bb.count] = blocks;
            if (a.pairs && !a.delay_mode) {  // one staging-buffer size: the largest
                int sb = 0;
                for (int k = 0; k < bb.count; ++k) sb = std::max(sb, bb.e[k].stage_bytes);
                for (int k = 0; k < bb.count; ++k) bb.e[k].stage_bytes = sb;
                smem = 128 + 2 * (size_t)sb;
            }
            e = kBeamBatchLaunchers[a.order](bb, a.delay_mode, a.chan_prec, a.ng_prec, blocks,
                                             smem, s);
            if (e != cudaSuccess) return cuda_fail(v[cls[b0]].plan, e, "beamform batch");
        }
    }
    // K3: envelope, grouped by identical taps and by engine (CUDA-core FIR for
    // small frames, tensor cores otherwise)
    std::fill(done.begin(), done.end(), false);
    for (size_t i = 0; i < v.size(); ++i) {
        if (done[i] || v[i].plan->hp.L == 0) continue;
        const HostPlan &a = v[i].plan->hp;
        const bool fir = env_on_cuda_cores(v[i].plan);
        std::vector<size_t> cls;
        for (size_t j = i; j < v.size(); ++j) {
            const HostPlan &b = v[j].plan->hp;
            if (!done[j] && b.L == a.L && b.taps == a.taps &&
                env_on_cuda_cores(v[j].plan) == fir) {
                cls.push_back(j);
                done[j] = true;
            }
        }
        for (size_t b0 = 0; fir && b0 < cls.size(); b0 += kBatchMax) {
            EnvFirParams fp{};
            fp.count = (int)std::min<size_t>(kBatchMax, cls.size() - b0);
            unsigned ctas = 0;
            for (int k = 0; k < fp.count; ++k) {
                const BatchEntry &x = v[cls[b0 + k]];
                fp.job[k] = fir_job(x.plan, x.ybuf, x.image, ctas);
                ctas += fir_ctas(x.plan);
            }
            fp.H = (a.L - 1) / 2;
            fp.taps = v[cls[b0]].plan->d_taps;
            fp.err = v[cls[b0]].plan->d_err;
            envelope_fir_kernel<<<ctas, kFirTile, 0, s>>>(fp);
            if ((e = cudaGetLastError()) != cudaSuccess)
                return cuda_fail(v[cls[b0]].plan, e, "envelope fir batch");
        }
        for (size_t b0 = 0; !fir && b0 < cls.size(); b0 += kBatchMax) {
            EnvTcParams ep{};
            ep.count = (int)std::min<size_t>(kBatchMax, cls.size() - b0);
            unsigned tiles = 0;
            for (int k = 0; k < ep.count; ++k) {
                const BatchEntry &x = v[cls[b0 + k]];
                ep.job[k] = env_job(x.plan, x.ybuf, x.image, tiles);
                tiles += env_tiles(x.plan);
            }
            const dmas_plan *pa = v[cls[b0]].plan;
            ep.total_tiles = tiles;
            ep.H = (a.L - 1) / 2;
            ep.n_stages = env_tc_stages(a);
            ep.taps = pa->d_taps_tc;
            ep.err = pa->d_err;
            int cap = 0;  // the smallest cap any entry asks for
            for (int k = 0; k < ep.count; ++k) {
                const int c = v[cls[b0 + k]].plan->env_tile_cap;
                if (c > 0 && (cap == 0 || c < cap)) cap = c;
            }
            e = launch_env_tc(ep, env_grid(tiles, pa->num_sms, cap), pa->smem_env, s);
            if (e != cudaSuccess) return cuda_fail(v[cls[b0]].plan, e, "envelope batch");
        }
    }
    return DMAS_OK;
}

// The every-order pass: matched filter (if the plan has one), root planes,
// one every-order beamform launch into `n_img` images (or their pre-envelope
// copies), and one envelope launch over all of them.
dmas_status enqueue_orders(dmas_plan *p, const float *d_frame, unsigned mask, int variants,
                           float *d_images, float *d_cf, cudaStream_t s) {
    const HostPlan &hp = p->hp;
    OrdersParams op;
    std::memset(&op, 0, sizeof(op));
    int n_img = 0;
    for (int v = 0; v < 2; ++v)
        for (int k = 0; k <= kOrdersMaxOrder; ++k)
            op.slot[v][k] = (k >= 1 && ((variants >> v) & 1) && ((mask >> (k - 1)) & 1))
                                ? n_img++
                                : -1;
    const size_t plane = (size_t)hp.N * hp.row;
    const int n_planes = orders_planes(hp.order);
    const size_t chan_b = align256(sizeof(float) * plane * n_planes);
    const size_t img = (size_t)hp.M * hp.T;
    const size_t y_b = hp.L > 0 ? align256(sizeof(float) * img * n_img) : 0;
    const size_t need = chan_b + y_b + align256(p->mf_bytes);
    cudaError_t e;
    if (need > p->orders_bytes) {
        cudaFree(p->d_orders);  // waits for work still using the old buffer
        p->d_orders = nullptr;
        p->orders_bytes = 0;
        if ((e = cudaMalloc(&p->d_orders, need)) != cudaSuccess) {
            cudaGetLastError();
            p->last_error = "every-order scratch: " + std::string(cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? DMAS_ENOMEM : DMAS_ECUDA;
        }
        p->orders_bytes = need;
    }
    char *base = (char *)p->d_orders;
    float *chan = (float *)base;
    float *ybuf = hp.L > 0 ? (float *)(base + chan_b) : d_images;
    mark(p, 0, s);
    if (!hp.mf.empty()) {
        MfParams mp{};
        mp.count = 1;
        mp.job[0] = mf_job(p, d_frame, p->d_scratch, 0);
        mp.job[0].out = (float *)(base + chan_b + y_b);
        e = launch_mf(mp, mf_ctas(p), sizeof(float) * mf_smem_floats(mp.job[0].L), s);
        if (e != cudaSuccess) return cuda_fail(p, e, "matched_filter_kernel launch");
        d_frame = mp.job[0].out;
    }
    RootPlanesParams rp;
    rp.frame = d_frame;
    rp.chan = chan;
    rp.plane = plane;
    rp.N = hp.N;
    rp.T = hp.T;
    rp.row = hp.row;
    rp.padl = hp.padl;
    const unsigned rgrid = roots_blocks(p);
    switch (hp.order) {
        case 1: root_planes_kernel<1><<<rgrid, 256, 0, s>>>(rp); break;
        case 2: root_planes_kernel<2><<<rgrid, 256, 0, s>>>(rp); break;
        case 3: root_planes_kernel<3><<<rgrid, 256, 0, s>>>(rp); break;
        case 4: root_planes_kernel<4><<<rgrid, 256, 0, s>>>(rp); break;
        default: root_planes_kernel<5><<<rgrid, 256, 0, s>>>(rp); break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(p, e, "root_planes_kernel launch");
    mark(p, 1, s);

    op.chan = chan;
    op.plane = plane;
    op.use_tma = 0;
    if (hp.mo_window <= kTmaMaxBox) {
        if (EncodeTiledFn enc = encode_tiled()) {
            // planes [n_planes][N][row]: one box per microphone, its window
            // of every plane
            cuuint64_t dims[3] = {(cuuint64_t)hp.row, (cuuint64_t)hp.N, (cuuint64_t)n_planes};
            cuuint64_t strides[2] = {(cuuint64_t)hp.row * 4, (cuuint64_t)plane * 4};
            cuuint32_t box[3] = {(cuuint32_t)hp.mo_window, 1, (cuuint32_t)n_planes};
            cuuint32_t es[3] = {1, 1, 1};
            if (enc(&op.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)chan, dims, strides, box,
                    es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
                op.use_tma = 1;
        }
    }
    op.gdir = p->d_gdir;
    op.gws = p->d_gws;
    op.rel = p->d_rel;
    op.wf2 = p->d_wf2;
    op.y = ybuf;
    op.img = img;
    op.cf = d_cf;
    op.err = p->d_err;
    op.N = hp.N;
    op.T = hp.T;
    op.row = hp.row;
    op.padl = hp.padl;
    op.window = hp.mo_window;
    op.halves = hp.mo_halves;
    op.mic_chunk = hp.mo_chunk;
    op.n_groups = hp.n_groups;
    op.n_mics_f = (float)hp.N;
    op.cf_eps = (float)hp.cf_eps;
    const bool lin = hp.delay_mode == DMAS_DELAY_LINEAR;
    e = kOrdersLaunchers[hp.order](op, lin ? 1 : 0, hp.ng_prec,
                                   (unsigned)((size_t)hp.n_groups * hp.mo_tiles),
                                   orders_smem_bytes(hp.order, lin, hp.mo_chunk, hp.mo_window,
                                                     hp.mo_halves),
                                   s);
    if (e != cudaSuccess) return cuda_fail(p, e, "beamform_orders_kernel launch");
    mark(p, 2, s);
    p->env_ran = hp.L > 0;
    if (hp.L > 0) {
        // the plan's envelope engine (chosen by its M), so an image does not
        // depend on how many others the call asked for
        const int rows = hp.M * n_img;
        if (env_on_cuda_cores(p)) {
            EnvFirParams fp{};
            fp.count = 1;
            fp.H = (hp.L - 1) / 2;
            fp.taps = p->d_taps;
            fp.err = p->d_err;
            fp.job[0] = fir_job(p, ybuf, d_images, 0, rows);
            envelope_fir_kernel<<<fir_ctas(p, rows), kFirTile, 0, s>>>(fp);
            if ((e = cudaGetLastError()) != cudaSuccess)
                return cuda_fail(p, e, "envelope_fir_kernel launch");
        } else {
            EnvTcParams ep{};
            ep.count = 1;
            ep.job[0] = env_job(p, ybuf, d_images, 0, rows);
            ep.total_tiles = env_tiles(p, rows);
            ep.H = (hp.L - 1) / 2;
            ep.n_stages = env_tc_stages(hp);
            ep.taps = p->d_taps_tc;
            ep.err = p->d_err;
            e = launch_env_tc(ep, env_grid(ep.total_tiles, p->num_sms, p->env_tile_cap),
                              p->smem_env, s);
            if (e != cudaSuccess) return cuda_fail(p, e, "envelope_tc_kernel launch");
        }
    }
    mark(p, 3, s);
    p->profiled_once = p->profiled_once || p->profiling;
    return DMAS_OK;
}

}  // namespace

extern "C" {

int dmas_version(void) { return 100; }

const char *dmas_status_string(dmas_status s) {
    switch (s) {
        case DMAS_OK: return "ok";
        case DMAS_EINVAL: return "invalid argument";
        case DMAS_ENOMEM: return "out of memory";
        case DMAS_ECUDA: return "CUDA error";
        case DMAS_EBUSY: return "busy";
        case DMAS_ETIMEOUT: return "device wait timed out";
        case DMAS_EBOUNDS: return "kernel index out of bounds (host-checked build)";
    }
    return "unknown status";
}

dmas_status dmas_plan_create(const dmas_plan_desc *desc, dmas_plan **out) {
    if (!out) return DMAS_EINVAL;
    *out = nullptr;
    if (!desc) return DMAS_EINVAL;
    dmas_plan *p = new (std::nothrow) dmas_plan();
    if (!p) return DMAS_ENOMEM;
    std::string why;
    dmas_status st;
    try {
        st = build_host_plan(*desc, p->hp, &why);
    } catch (const std::bad_alloc &) {
        delete p;
        return DMAS_ENOMEM;
    }
    if (st != DMAS_OK) {
        delete p;
        return st;
    }
    HostPlan &hp = p->hp;
    cudaGetDevice(&p->device);
    if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) !=
            cudaSuccess ||
        p->num_sms < 1)
        p->num_sms = 148;
    cudaGetLastError();
    p->smem_beam = beam_smem_bytes(hp);
    p->smem_env = env_smem_bytes(hp);
    cudaError_t e;
    if ((e = upload(&p->d_gdir, hp.gdir)) != cudaSuccess ||
        (e = upload(&p->d_gws, hp.gws)) != cudaSuccess ||
        (e = upload(&p->d_rel, hp.rel)) != cudaSuccess ||
        (e = upload(&p->d_frac, hp.gfrac)) != cudaSuccess ||
        (e = upload(&p->d_sel, hp.gsel)) != cudaSuccess ||
        (e = upload(&p->d_wf2, hp.gwf2)) != cudaSuccess) {
        free_plan_memory(p);
        delete p;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? DMAS_ENOMEM : DMAS_ECUDA;
    }
    if (hp.L > 0) {
        std::vector<float> tc;
        try {
            tc = tc_tap_arrays(hp);
        } catch (const std::bad_alloc &) {
            free_plan_memory(p);
            delete p;
            return DMAS_ENOMEM;
        }
        if ((e = upload(&p->d_taps_tc, tc)) != cudaSuccess ||
            (e = upload(&p->d_taps, hp.taps)) != cudaSuccess) {
            free_plan_memory(p);
            delete p;
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? DMAS_ENOMEM : DMAS_ECUDA;
        }
    }
    p->table_bytes = (hp.gdir.size() + hp.gws.size() + hp.rel.size() + hp.gfrac.size() +
                      hp.gsel.size() + hp.gwf2.size()) * 4;
    // the interpolated-delay pair kernel also reads the raw samples as a
    // second zero-padded plane
    p->chan_bytes = (size_t)hp.N * hp.row * chan_elem_bytes(hp.chan_prec) *
                    (uses_raw_rows(hp.chan_prec, hp.order, hp.delay_mode) ? 2 : 1);
    p->ybuf_bytes = hp.L > 0 ? sizeof(float) * (size_t)hp.M * hp.T : 0;
    p->mf_bytes = hp.mf.empty() ? 0 : sizeof(float) * (size_t)hp.N * hp.T;
    if (!hp.mf.empty() && (e = upload(&p->d_mf, hp.mf)) != cudaSuccess) {
        free_plan_memory(p);
        delete p;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? DMAS_ENOMEM : DMAS_ECUDA;
    }
    if ((e = cudaMalloc((void **)&p->d_err, 256)) != cudaSuccess ||
        (e = cudaMemset(p->d_err, 0, 256)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_scratch, scratch_bytes(p))) !=
            cudaSuccess) {
        free_plan_memory(p);
        delete p;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? DMAS_ENOMEM : DMAS_ECUDA;
    }
    *out = p;
    return DMAS_OK;
}

dmas_status dmas_destroy(dmas_plan *p) {
    if (!p) return DMAS_OK;
    cudaDeviceSynchronize();
    free_plan_memory(p);
    delete p;
    return DMAS_OK;
}

size_t dmas_plan_workspace_bytes(const dmas_plan *p) {
    if (!p) return 0;
    return scratch_bytes(p);
}

dmas_status dmas_beamform(dmas_plan *p, const float *d_frame, float *d_image, float *d_y,
                          float *d_cf, void *stream) {
    if (!p || !d_frame || !d_image) return DMAS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    return enqueue_frame(p, d_frame, d_image, d_y, d_cf, p->d_scratch, s);
}

dmas_status dmas_beamform_orders(dmas_plan *p, const float *d_frame, unsigned orders_mask,
                                 int variants, float *d_images, float *d_cf, void *stream) {
    if (!p || !d_frame || !d_images) return DMAS_EINVAL;
    const HostPlan &hp = p->hp;
    if (hp.mo_chunk == 0) {
        p->last_error = "dmas_beamform_orders: the plan needs FP32 channels, order <= 5 and a "
                        "delay spread whose staged windows fit in shared memory";
        return DMAS_EINVAL;
    }
    if (orders_mask == 0 || (orders_mask >> hp.order) != 0) {
        p->last_error = "dmas_beamform_orders: orders_mask must select orders in 1..order";
        return DMAS_EINVAL;
    }
    if (variants < DMAS_V_PLAIN || variants > (DMAS_V_PLAIN | DMAS_V_CF)) {
        p->last_error = "dmas_beamform_orders: variants must be DMAS_V_PLAIN, DMAS_V_CF or both";
        return DMAS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    return enqueue_orders(p, d_frame, orders_mask, variants, d_images, d_cf, s);
}

dmas_status dmas_beamform_host(dmas_plan *p, const float *h_frame, float *h_image,
                               void *stream) {
    if (!p || !h_frame || !h_image) return DMAS_EINVAL;
    const HostPlan &hp = p->hp;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t fbytes = sizeof(float) * (size_t)hp.N * hp.T;
    const size_t ibytes = sizeof(float) * (size_t)hp.M * hp.T;
    cudaError_t e;
    if (!p->d_io_frame && cudaMalloc((void **)&p->d_io_frame, fbytes) != cudaSuccess) {
        p->d_io_frame = nullptr;
        cudaGetLastError();
        return DMAS_ENOMEM;
    }
    if (!p->d_io_image && cudaMalloc((void **)&p->d_io_image, ibytes) != cudaSuccess) {
        p->d_io_image = nullptr;
        cudaGetLastError();
        return DMAS_ENOMEM;
    }
    if (!p->copy_stream) {
        if ((e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking)) !=
            cudaSuccess) {
            p->copy_stream = nullptr;
            return cuda_fail(p, e, "copy stream");
        }
        for (auto &ev : p->chunk_ev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
                ev = nullptr;
                return cuda_fail(p, e, "chunk events");
            }
    }
    p->last_stream = s;
    if ((e = cudaMemcpyAsync(p->d_io_frame, h_frame, fbytes, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return cuda_fail(p, e, "frame upload");
    dmas_status st =
        enqueue_host_chunks(p, p->d_io_frame, p->d_io_image, h_image, p->d_scratch, s);
    if (st != DMAS_OK) return st;
    if ((e = cudaStreamSynchronize(p->copy_stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(p, e, "synchronise");
    return DMAS_OK;
}

size_t dmas_batch_workspace_bytes(int count, dmas_plan *const *plans) {
    if (count < 1 || !plans) return 0;
    size_t total = 0;
    for (int k = 0; k < count; ++k) {
        if (!plans[k]) return 0;
        total += dmas_plan_workspace_bytes(plans[k]);
    }
    return total;
}

dmas_status dmas_beamform_batch(int count, dmas_plan *const *plans, const float *const *d_frames,
                                float *const *d_images, void *d_workspace, size_t workspace_bytes,
                                void *stream) {
    if (count < 1 || !plans || !d_frames || !d_images || !d_workspace) return DMAS_EINVAL;
    for (int k = 0; k < count; ++k)
        if (!plans[k] || !d_frames[k] || !d_images[k]) return DMAS_EINVAL;
    if (((uintptr_t)d_workspace & 255) != 0) return DMAS_EINVAL;
    if (workspace_bytes < dmas_batch_workspace_bytes(count, plans)) return DMAS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // A batch of one runs exactly as dmas_beamform runs it, on the workspace:
    // the batch kernels find each CTA's entry and normalise the staging size
    // across entries, which a lone frame does not need (measured on B300, one
    // 128 x 8192 x 32768 frame: 8.49 ms as a batch, 8.23 ms alone).
    if (count == 1) {
        plans[0]->last_stream = s;
        return enqueue_frame(plans[0], d_frames[0], d_images[0], nullptr, nullptr, d_workspace,
                             s);
    }
    char *ws = (char *)d_workspace;
    std::vector<BatchEntry> v;
    try {
        v.reserve(count);
    } catch (const std::bad_alloc &) {
        return DMAS_ENOMEM;
    }
    for (int k = 0; k < count; ++k) {
        plans[k]->last_stream = s;
        BatchEntry x;
        x.plan = plans[k];
        x.frame = d_frames[k];
        x.image = d_images[k];
        x.scratch = ws;
        x.ybuf = y_target(plans[k], d_images[k], nullptr, ws);
        v.push_back(x);
        ws += dmas_plan_workspace_bytes(plans[k]);
    }
    return enqueue_batch(v, s);
}

dmas_status dmas_beamform_batch_upload(int count, dmas_plan *const *plans,
                                       const float *const *h_frames, float *const *d_frames,
                                       float *const *d_images, void *d_workspace,
                                       size_t workspace_bytes, void *stream, void *done_event) {
    if (count < 1 || !plans || !h_frames || !d_frames) return DMAS_EINVAL;
    for (int k = 0; k < count; ++k)
        if (!plans[k] || !h_frames[k] || !d_frames[k]) return DMAS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < count; ++k) {
        const size_t bytes = (size_t)plans[k]->hp.N * plans[k]->hp.T * sizeof(float);
        const cudaError_t e =
            cudaMemcpyAsync(d_frames[k], h_frames[k], bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(plans[k], e, "frame upload");
    }
    const dmas_status st =
        dmas_beamform_batch(count, plans, d_frames, d_images, d_workspace, workspace_bytes, stream);
    if (st != DMAS_OK || !done_event) return st;
    const cudaError_t e = cudaEventRecord((cudaEvent_t)done_event, s);
    return e == cudaSuccess ? DMAS_OK : cuda_fail(plans[0], e, "completion event");
}

dmas_status dmas_plan_get_info(const dmas_plan *p, dmas_plan_info *info) {
    if (!p || !info) return DMAS_EINVAL;
    const HostPlan &hp = p->hp;
    info->n_mics = hp.N;
    info->n_dirs = hp.M;
    info->n_samples = hp.T;
    info->order = hp.order;
    info->delay_mode = hp.delay_mode;
    info->flags = hp.flags;
    info->chan_prec = hp.chan_prec;
    info->ng_prec = hp.ng_prec;
    info->env_taps = hp.L;
    info->n_groups = hp.n_groups;
    info->group_size = kGroup;
    info->window = hp.window;
    info->mic_chunk = hp.mic_chunk;
    info->time_tile = hp.tile;
    info->row = hp.row;
    info->workspace_bytes = dmas_plan_workspace_bytes(p);
    info->table_bytes = p->table_bytes;
    return DMAS_OK;
}

dmas_status dmas_plan_get_delays(const dmas_plan *p, int32_t *shift, float *frac) {
    if (!p || !shift) return DMAS_EINVAL;
    std::memcpy(shift, p->hp.shift.data(), p->hp.shift.size() * sizeof(int32_t));
    if (frac) std::memcpy(frac, p->hp.frac.data(), p->hp.frac.size() * sizeof(float));
    return DMAS_OK;
}

dmas_status dmas_plan_get_taps(const dmas_plan *p, float *taps) {
    if (!p || !taps) return DMAS_EINVAL;
    if (p->hp.L > 0) std::memcpy(taps, p->hp.taps.data(), sizeof(float) * p->hp.L);
    return DMAS_OK;
}

dmas_status dmas_plan_check(dmas_plan *p) {
    if (!p) return DMAS_EINVAL;
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "synchronise");
    unsigned word = 0;
    if ((e = cudaMemcpy(&word, p->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(p, e, "error word read");
    if (word) {
        cudaMemset(p->d_err, 0, sizeof(unsigned));
        if (word & kErrBounds) {
            p->last_error = "a kernel index fell outside its buffer (host-checked build)";
            return DMAS_EBOUNDS;
        }
        p->last_error = "a device wait timed out";
        return DMAS_ETIMEOUT;
    }
    return DMAS_OK;
}

const char *dmas_plan_last_error(const dmas_plan *p) {
    if (!p) return "";
    return p->last_error.c_str();
}

dmas_status dmas_plan_set_envelope_tile_cap(dmas_plan *p, int tiles_per_cta) {
    if (!p || tiles_per_cta < 0) return DMAS_EINVAL;
    p->env_tile_cap = tiles_per_cta;
    return DMAS_OK;
}

dmas_status dmas_plan_set_profiling(dmas_plan *p, int enable) {
    if (!p) return DMAS_EINVAL;
    if (enable && !p->ev[0]) {
        for (auto &e : p->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_fail(p, r, "event create");
        }
    }
    p->profiling = enable != 0;
    return DMAS_OK;
}

dmas_status dmas_plan_stage_ms(dmas_plan *p, float *roots_ms, float *beam_ms, float *env_ms) {
    if (!p || !p->profiled_once || !p->ev[0]) return DMAS_EINVAL;
    cudaError_t e = cudaEventSynchronize(p->ev[3]);
    if (e != cudaSuccess) return cuda_fail(p, e, "event synchronise");
    float t[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
        e = cudaEventElapsedTime(&t[k], p->ev[k], p->ev[k + 1]);
        if (e != cudaSuccess) return cuda_fail(p, e, "event elapsed");
    }
    if (roots_ms) *roots_ms = t[0];
    if (beam_ms) *beam_ms = t[1];
    if (env_ms) *env_ms = p->env_ran ? t[2] : 0.0f;
    return DMAS_OK;
}

dmas_status dmas_selftest_wait_timeout(double limit_ms, void *stream) {
    if (!(limit_ms >= 1.0 && limit_ms <= 10000.0)) return DMAS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *d_err = nullptr;
    cudaError_t e = cudaMalloc((void **)&d_err, sizeof(unsigned));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? DMAS_ENOMEM : DMAS_ECUDA;
    }
    unsigned word = 0;
    if ((e = cudaMemsetAsync(d_err, 0, sizeof(unsigned), s)) == cudaSuccess) {
        wait_timeout_selftest_kernel<<<1, 32, 0, s>>>(
            d_err, (unsigned long long)(limit_ms * 1.0e6));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&word, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_err);
    if (e != cudaSuccess) return DMAS_ECUDA;
    return word ? DMAS_ETIMEOUT : DMAS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Beamforming without any device allocation: the scratch lives in a static
// device array that the library holds on every GPU it is loaded on.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[DMAS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kMaxDevices] = {};

// The array's name in host code is only a stand-in; the device address comes
// from the runtime, looked up once per device with that device current.
dmas_status noalloc_scratch_address(int device, void **addr, std::string *why) {
    if (device < 0 || device >= kMaxDevices) {
        *why = "device ordinal out of range for the static scratch table";
        return DMAS_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            *why = std::string("cudaGetSymbolAddress of the static scratch: ") +
                   cudaGetErrorString(e);
            cudaGetLastError();
            return DMAS_ECUDA;
        }
        g_noalloc_addr[device] = p;
    }
    *addr = g_noalloc_addr[device];
    return DMAS_OK;
}

}  // namespace

extern "C" dmas_status dmas_beamform_noalloc(dmas_plan *p, const float *d_frame, float *d_image,
                                             void *stream) {
    if (!p || !d_frame || !d_image) return DMAS_EINVAL;
    const size_t need = dmas_plan_workspace_bytes(p);
    if (need > DMAS_NOALLOC_SCRATCH_BYTES) {
        p->last_error = "dmas_beamform_noalloc: this plan needs " + std::to_string(need) +
                        " bytes of scratch, more than the static " +
                        std::to_string((size_t)DMAS_NOALLOC_SCRATCH_BYTES) +
                        "-byte array; use dmas_beamform";
        return DMAS_EINVAL;
    }
    int device = -1;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaGetDevice");
    if (device != p->device) {
        p->last_error = "dmas_beamform_noalloc: the plan belongs to device " +
                        std::to_string(p->device) + " but device " + std::to_string(device) +
                        " is current";
        return DMAS_EINVAL;
    }
    void *scratch = nullptr;
    std::string why;
    dmas_status st = noalloc_scratch_address(device, &scratch, &why);
    if (st != DMAS_OK) {
        p->last_error = why;
        return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    // The roots stage rewrites the whole channel region, zero pads included,
    // and the beamform stage writes every y sample the envelope reads, so
    // nothing from an earlier call survives into this one.
    return enqueue_frame(p, d_frame, d_image, nullptr, nullptr, scratch, s);
}
