// Envelope low-pass on the tensor cores (tcgen05, kind::tf32).
//
// The FIR  e[d][t] = sum_x g[x] |y[d][t - H + x]|  (g the symmetric taps,
// x = 0..2H) is, for a tile of 128 direction rows and J = 128 output samples
// starting at t0, the product  E[128][J] = A[128][K] . B[K][J]  with
//   A[m][u] = |y[d0 + m][t0 - HA + u]|        (u = 0..K-1, K = J + 2 HA)
//   B[u][j] = g~[u - j]                        (a band: the taps slid by j)
// where HA = H rounded up to 4 (so every load starts 16-byte aligned) and g~ is
// g shifted by HA - H and zero outside the taps.  A is K-major (rows of y are
// contiguous in t).  B is K-major too.  The J outputs are issued as four MMAs
// of N = 32 columns each, in one of two forms:
//
//  * Toeplitz blocks (filters up to 209 taps): block b covers the consecutive
//    outputs j = 32 b + n (n = 0..31), whose band is only the 32 + 2 HA rows
//    u = 32 b + u' (u' = 0..31 + 2 HA) of B, where B[u][j] = T[u'][n] =
//    g~[u' - n] -- the same matrix T for every block.  T (hi and lo parts) is
//    stored once per CTA in the canonical K-major layout (core matrices of
//    8 columns x 4 rows, 128 bytes; K-adjacent core matrices 128 bytes apart,
//    8-column groups 32 (32 + 2 HA) bytes apart), so block b's MMA at tile
//    k-step s reads T from row 8 s - 32 b.  Each block multiplies 32 + 2 HA
//    rows of K instead of the tile's whole J + 2 HA: for 181 taps 216 of 312
//    (27 of 39 k-steps), and its columns are outputs in order.
//  * Phases (longer filters, whose T does not fit beside the stages): a
//    shared-memory matrix descriptor can only step rows by 16 bytes (4 samples),
//    so the outputs are taken as 4 phases r (j = 4q + r), and phase r's J/4
//    columns, in reverse order of q, are rows of a tap array that step by
//    exactly 16 bytes -- one descriptor over one array per phase, no matrix
//    materialised, every MMA over the tile's whole K.  Phase r accumulates into
//    TMEM columns [r J/4, (r + 1) J/4).  Measured on B300 in this form, J = 128
//    is the fastest tile (J = 256: 131 us, 192: 120 us, 128: 110 us, 64: 161 us
//    for a 2048 x 16384 frame).
//
// FP32 accuracy from TF32 products: A = A_hi + A_lo and g = g_hi + g_lo with
// the _hi parts rounded to TF32; each k-step issues A_hi.B_hi + A_hi.B_lo +
// A_lo.B_hi (the dropped A_lo.B_lo term is ~2^-22 relative).
//
// The split |y| (A_hi, A_lo) is the MMA's A operand in tensor memory, so
// shared memory feeds the tensor core only the taps (B): with A in shared
// memory, the four phases x three products re-read the same A twelve times per
// k-step and shared-memory bandwidth bound the kernel (L1 79 % busy).
//
// |y| is staged in the K-major layout with the 128-byte swizzle: for each
// 32-sample column of a k-block ("atom"), row m occupies bytes
// [128 m, 128 m + 128) and its 16-byte chunk c (samples 4c..4c+3) sits at
// chunk position c ^ (m & 7); TMA writes it directly from 128-byte rows of y
// and the split pass reads a row per thread without bank conflicts.
//
// CTA: 13 warps, persistent over tiles (and over the frames of a batch), with
// warp roles: a producer stages each k-block of 64 samples of y by TMA (2-D
// tensor map, two boxes of 32 samples x 128 rows; cp.async to the same layout
// when T % 4 != 0) into one of n_stages shared-memory stages (up to
// kTcStages: as many as fit beside the tap operand); 4 split warps (one row
// per thread, the warp's TMEM lane quarter) read |y| rounded to TF32 and the
// remainder and store them (tcgen05.st) into an A stage in TMEM (hi, lo:
// 2 x 64 columns); four MMA warps (one block or phase each) issue the
// k-block's k-steps x 3 MMAs and commit them to the A stage's mbarrier.
//  * Toeplitz form: one accumulator (J columns from column 0) with a full and
//    an empty barrier per block, three A stages after it.  A block's warp
//    commits its block's full barrier after the block's last k-step; the
//    epilogue reads the block's 32 columns, hands them back (empty barrier),
//    writes the row's 32 outputs into a 128-byte swizzled shared-memory buffer
//    and one thread stores the 32 x 128 box with a tensor store (two buffers
//    alternate; a buffer is rewritten only after its store has read it).
//  * Phase form: two accumulators (2 x J columns), two A stages after them;
//    the epilogue reads a finished accumulator while the next tile
//    accumulates into the other and stores 8 consecutive outputs (one 32-byte
//    sector) at a time.
// Every wait is bounded.
#pragma once

#include <cuda.h>

#include "dmas_kernels.cuh"

namespace dmas {

constexpr int kTcRows = 128;         // direction rows per tile (MMA M)
constexpr int kTcJ = 128;            // output samples per tile
constexpr int kTcNq = kTcJ / 4;      // columns per phase (MMA N)
constexpr int kTcKB = 64;            // samples per k-block
constexpr int kTcAtomK = 32;         // samples per 128-byte swizzle atom column
constexpr int kTcAtomBytes = kTcRows * 128;  // one atom column of 128 rows
constexpr int kTcBufBytes = kTcRows * kTcKB * 4;  // one of A_hi / A_lo for a k-block

constexpr int kTcStageBytes = kTcBufBytes;  // |y| of one k-block, FP32
constexpr int kTcStages = 6;  // most shared-memory stages (fewer for long filters)
// dynamic shared memory the kernel may take (it also has ~1 KB of static)
constexpr int kEnvSmemMax = 222 * 1024;

__host__ __device__ inline int tc_halo(int H) { return (H + 3) & ~3; }
__host__ __device__ inline int tc_K(int H) { return kTcJ + 2 * tc_halo(H); }
// length of one phase tap array (floats), a multiple of 8
__host__ __device__ inline int tc_Z(int H) { return (tc_K(H) + 4 * (kTcNq - 1) + 7) & ~7; }
// rows of the Toeplitz block matrix T (the K one block of 32 outputs spans)
__host__ __device__ inline int tc_KB(int H) { return kTcNq + 2 * tc_halo(H); }
// bytes of the tap operand in shared memory: T hi and lo, 32 columns x KB
// rows of 4 bytes each; or the 8 phase arrays
__host__ __device__ inline int tc_toep_bytes(int H) { return 2 * 32 * 4 * tc_KB(H); }
__host__ __device__ inline int tc_phase_bytes(int H) { return 8 * 4 * tc_Z(H); }
__host__ __device__ inline int tc_align1k(int b) { return (b + 1023) & ~1023; }
// The Toeplitz form whenever T and the two store buffers leave room for 4
// stages of |y|
__host__ __device__ inline bool tc_toeplitz(int H) {
    return kEnvSmemMax - 1024 - tc_align1k(tc_toep_bytes(H)) - 2 * kTcRows * kTcNq * 4 >=
           4 * kTcStageBytes;
}
__host__ __device__ inline int tc_tap_bytes(int H) {
    return tc_toeplitz(H) ? tc_toep_bytes(H) : tc_phase_bytes(H);
}
// Toeplitz form: two store buffers (one block of 32 outputs x 128 rows each,
// 128-byte swizzled) between the epilogue and the tensor stores
constexpr int kTcOutBytes = kTcRows * kTcNq * 4;
__host__ __device__ inline int tc_out_bytes(int H) { return tc_toeplitz(H) ? 2 * kTcOutBytes : 0; }

struct EnvTcJob {
    // 2-D view of y for the TMA engine when T % 4 == 0: dims (T, M), box
    // {32 samples, 128 rows} with the 128-byte swizzle, landing as one atom
    // column of A; out-of-range coordinates filled with zeros.
    CUtensorMap tmap;
    // 2-D view of the image for tensor stores (Toeplitz form): dims (T, M),
    // box {32 outputs, 128 rows}, 128-byte swizzle; valid when use_tma_store
    CUtensorMap omap;
    const float *y;   // [M][T]
    float *img;       // [M][T]
    int M, T;
    int tt0;          // first time tile (kTcJ outputs) of this job
    int t_tiles;      // time tiles of this job (all: ceil(T / kTcJ))
    int use_tma;      // T % 4 == 0 and the map was encoded
    int use_tma_store;  // T % 4 == 0, img 16-byte aligned and omap encoded
    unsigned first;   // first tile of this job in the launch
};

struct EnvTcParams {
    int count;
    unsigned total_tiles;
    int H;
    int n_stages;       // shared-memory stages of |y|, 2..kTcStages
    // the tap operand, tc_tap_bytes(H) bytes (device): T hi then T lo in the
    // Toeplitz form's core-matrix layout, else the phase arrays [2][4][Z]
    const float *taps;
    unsigned *err;
    EnvTcJob job[kBatchMax];
};
static_assert(sizeof(EnvTcParams) <= 32764, "kernel parameters exceed the launch limit");

// Shared-memory matrix descriptor: start, leading and stride byte offsets,
// version 1 (sm_100 family), base offset 0, layout (0 = no swizzle, 2 = the
// 128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo,
                                              uint32_t layout = 0) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)layout << 61;
    return d;
}

// byte offset of row m's 16-byte chunk c (c = 0..15 over a k-block) in the
// swizzled A buffer of a stage
__device__ __forceinline__ int sw128_off(int m, int c) {
    return (c >> 3) * kTcAtomBytes + m * 128 + (((c & 7) ^ (m & 7)) << 4);
}

// kind::tf32 instruction descriptor: D f32, A/B tf32, both K-major, N and M.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
// make `bar`'s phase wait for this thread's earlier cp.async copies (adds a
// pending arrival now, completes it when the copies have landed)
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}
// one 32-byte store (a whole L2 sector; p 32-byte aligned)
__device__ __forceinline__ void st_global_v8(float *p, float a, float b, float c, float d,
                                             float e, float f, float g, float h) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a),
                 "f"(b), "f"(c), "f"(d), "f"(e), "f"(f), "f"(g), "f"(h)
                 : "memory");
}

// tensor store of one box from shared memory (bulk-group completion)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int c0,
                                             int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map),
        "r"(smem_addr(src)), "r"(c0), "r"(c1)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// this thread's bulk groups but the newest N have finished reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// named barrier 1 over the 128 epilogue threads
__device__ __forceinline__ void epi_sync() {
    asm volatile("bar.sync 1, 128;" ::: "memory");
}
// named barrier 1 over the 128 epilogue threads, true iff every one passes true
__device__ __forceinline__ bool epi_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                     "r"(smem_addr(bar))
                 : "memory");
}

// Tile -> (job, row block, time tile).
struct TcTile {
    const EnvTcJob *job;
    int row0, t0;
};
__device__ __forceinline__ TcTile tc_tile(const EnvTcParams &p, unsigned tile) {
    int k = 0;
    while (k + 1 < p.count && p.job[k + 1].first <= tile) ++k;
    const EnvTcJob &jb = p.job[k];
    const unsigned local = tile - jb.first;
    const int rb = (int)(local / (unsigned)jb.t_tiles);
    const int tt = (int)(local - (unsigned)rb * (unsigned)jb.t_tiles);
    return {&jb, rb * kTcRows, (jb.tt0 + tt) * kTcJ};
}

// Warp roles: 0-3 split (one row each, TMEM lane quarters), 4-7 epilogue
// (TMEM lane quarters), 8 producer, 9.. MMA issue (lane 0 of each; warp 9 also
// allocates TMEM).  A tcgen05.mma costs its issuing thread tens of cycles, so
// the phases are spread over kTcMmaWarps issuing warps.
constexpr int kTcMmaWarps = 4;
constexpr int kTcPhasesPerWarp = 4 / kTcMmaWarps;
constexpr int kTcWarps = 9 + kTcMmaWarps;
constexpr int kTcThreadsWS = kTcWarps * 32;
constexpr uint32_t kTcAccCols = 4 * kTcNq;  // one accumulator (4 phases)
constexpr uint32_t kTcACol0 = 2 * kTcAccCols;  // first TMEM column of the A stages
constexpr uint32_t kTcACols = 2 * kTcKB;    // one A stage: hi then lo
constexpr int kTcAStages = (512 - (int)kTcACol0) / (int)kTcACols;  // A stages in TMEM
// Toeplitz form: one accumulator (J columns, block b at 32 b) with a full and
// an empty barrier per block, so a block's MMA warp starts the next tile as
// soon as the epilogue has read that block; the freed columns hold a third A
// stage, which lets the MMA warps drift apart by up to three k-blocks (their
// k-steps per k-block differ: each block's band covers a different part of K)
constexpr int kTcAStagesT = (512 - kTcJ) / (int)kTcACols;
constexpr int kTcAStagesMax = kTcAStagesT > kTcAStages ? kTcAStagesT : kTcAStages;

__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 32 consecutive TMEM columns of this thread's lane (warp-collective)
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
        "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]),
        "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]),
        "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]),
        "f"(v[29]), "f"(v[30]), "f"(v[31])
        : "memory");
}

template <bool TOEP>
__global__ void __launch_bounds__(kTcThreadsWS, 1)
    envelope_tc_kernel(const __grid_constant__ EnvTcParams p) {
    extern __shared__ __align__(128) unsigned char env_smem[];
    __shared__ uint64_t full[kTcStages], empty[kTcStages];
    __shared__ uint64_t a_full[kTcAStagesMax], a_empty[kTcAStagesMax], acc_full[4], acc_empty[4];
    // A stages and their first TMEM column, accumulator barriers
    constexpr int nA = TOEP ? kTcAStagesT : kTcAStages;
    constexpr uint32_t acol0 = TOEP ? (uint32_t)kTcJ : kTcACol0;
    constexpr int n_acc_bars = TOEP ? kTcMmaWarps : 2;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = p.H, HA = tc_halo(H), K = tc_K(H), Z = tc_Z(H);
    const int n_kb = (K + kTcKB - 1) / kTcKB;
    // the dynamic window starts 1024-aligned (its size has 1 KB to spare)
    unsigned char *base = env_smem + ((1024u - (smem_addr(env_smem) & 1023u)) & 1023u);
    const int tap_bytes = TOEP ? tc_toep_bytes(H) : tc_phase_bytes(H);
    float *s_taps = reinterpret_cast<float *>(base);  // T hi, T lo; or [2][4][Z]
    unsigned char *stages = base + tc_align1k(tap_bytes);  // [S]
    // Toeplitz form: the two store buffers after the stages (1024-aligned)
    unsigned char *obuf = stages + (size_t)p.n_stages * kTcStageBytes;
    // host-checked build: the taps and the stages inside the dynamic shared
    // memory (otherwise the CTA does no tile)
    const bool layout_ok =
        checked_ok(p.n_stages >= 2 && p.n_stages <= kTcStages &&
                       smem_in(s_taps, (uint32_t)tap_bytes) &&
                       smem_in(stages, (uint32_t)p.n_stages * (uint32_t)kTcStageBytes) &&
                       (!TOEP || smem_in(obuf, 2u * kTcOutBytes)),
                   p.err);
    const unsigned n_tiles = (layout_ok && blockIdx.x < p.total_tiles)
                                 ? (p.total_tiles - 1 - blockIdx.x) / gridDim.x + 1
                                 : 0;

    if (layout_ok)
        for (int i = tid; i < tap_bytes / 16; i += kTcThreadsWS)
            reinterpret_cast<float4 *>(s_taps)[i] = reinterpret_cast<const float4 *>(p.taps)[i];
    if (warp == 9) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < p.n_stages; ++s) {
            mbar_init(&full[s], 1);     // producer lane 0 (+ bytes or cp.async arrivals)
            mbar_init(&empty[s], 128);  // split threads, once they have read the stage
        }
        for (int a = 0; a < nA; ++a) {
            mbar_init(&a_full[a], 128);          // split threads, after their TMEM stores
            mbar_init(&a_empty[a], kTcMmaWarps); // MMA commits of the k-block that read it
        }
        for (int a = 0; a < n_acc_bars; ++a) {
            // MMA commits after a tile's last k-block (Toeplitz: the block's own warp)
            mbar_init(&acc_full[a], TOEP ? 1 : kTcMmaWarps);
            mbar_init(&acc_empty[a], 128);         // epilogue threads
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        if (abort_flag) return false;
        if (mbar_wait_bounded(bar, parity)) return true;
        abort_flag = 1;
        atomicOr(p.err, kErrTimeout);
        return false;
    };

    if (warp == 8) {
        // ------------------------------ producer -----------------------------
        unsigned g = 0;
        for (unsigned i = 0; i < n_tiles; ++i) {
            const TcTile tl = tc_tile(p, blockIdx.x + i * gridDim.x);
            const EnvTcJob &jb = *tl.job;
            for (int kb = 0; kb < n_kb; ++kb, ++g) {
                const int s = (int)(g % (unsigned)p.n_stages);
                const unsigned use = g / (unsigned)p.n_stages;
                if (use > 0 && !wait(&empty[s], (use - 1) & 1u)) goto done;
                float *ahi = reinterpret_cast<float *>(stages + (size_t)s * kTcStageBytes);
                const int u0 = kb * kTcKB;
                const int nc4 = min(kTcKB, K - u0) / 4;
                if (jb.use_tma) {
                    // two atom columns of 32 samples x 128 rows (32 KB); samples past
                    // K are loaded but never read by the MMAs
                    if (lane == 0) {
                        mbar_arrive_expect_tx(&full[s], (uint32_t)(kTcKB / kTcAtomK) * kTcAtomBytes);
                        // x = t0 - HA + u0 (+ 32): a multiple of 4 samples (16 bytes)
                        for (int a = 0; a < kTcKB / kTcAtomK; ++a)
                            tma_load_2d(reinterpret_cast<unsigned char *>(ahi) + a * kTcAtomBytes,
                                        &jb.tmap, tl.t0 - HA + u0 + kTcAtomK * a, tl.row0,
                                        &full[s]);
                    }
                    continue;
                }
                // fallback (T % 4 != 0): chunk (m, c), 4 samples of row m at
                // t = t0 - HA + u0 + 4c, copied to its swizzled position by 4-byte
                // cp.async with zero fill
                for (int idx = lane; idx < kTcRows * nc4; idx += 32) {
                    const int m = idx % kTcRows, c = idx / kTcRows;
                    const int row = tl.row0 + m;
                    const int t = tl.t0 - HA + u0 + 4 * c;
                    float *dst = ahi + (sw128_off(m, c) >> 2);
                    const float *rowp = jb.y + (size_t)(row < jb.M ? row : 0) * jb.T;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const bool in = row < jb.M && t + e >= 0 && t + e < jb.T;
                        cp_async4(dst + e, in ? rowp + t + e : jb.y, in ? 4u : 0u);
                    }
                }
                cp_async_arrive(&full[s]);
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[s]);
            }
        }
    } else if (warp < 4) {
        // ---------------------- split |y| -> hi, lo into TMEM ---------------
        const int m = tid;  // row of the tile = TMEM lane (warp w owns lanes 32w..)
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        unsigned g = 0;
        for (unsigned i = 0; i < n_tiles; ++i) {
            for (int kb = 0; kb < n_kb; ++kb, ++g) {
                const int s = (int)(g % (unsigned)p.n_stages);
                const int t = (int)(g % (unsigned)nA);
                const unsigned use = g / (unsigned)nA;
                if (!wait(&full[s], (g / (unsigned)p.n_stages) & 1u)) goto done;
                // the MMAs of the k-block nA back have finished reading A stage t
                if (use > 0 && !wait(&a_empty[t], (use - 1) & 1u)) goto done;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const float *ay = reinterpret_cast<const float *>(stages + (size_t)s * kTcStageBytes);
                const uint32_t acol = acol0 + (uint32_t)t * kTcACols;
#pragma unroll
                for (int half = 0; half < kTcKB / 32; ++half) {
                    float h[32], l[32];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float4 v = *reinterpret_cast<const float4 *>(
                            ay + (sw128_off(m, 8 * half + c) >> 2));
                        const float x[4] = {fabsf(v.x), fabsf(v.y), fabsf(v.z), fabsf(v.w)};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            h[4 * c + e] = tf32_round(x[e]);
                            l[4 * c + e] = x[e] - h[4 * c + e];
                        }
                    }
                    tmem_st32(lane_base + acol + (uint32_t)(32 * half), h);
                    tmem_st32(lane_base + acol + (uint32_t)(kTcKB + 32 * half), l);
                }
                // the stage has been read: order these reads before the
                // producer's next bulk copy into it
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&empty[s]);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&a_full[t]);
            }
        }
    } else if (warp >= 9) {
        // ------------------------------ MMA issue ----------------------------
        const int r0 = (warp - 9) * kTcPhasesPerWarp;  // this warp's phases
        const uint32_t idesc = tc_idesc(kTcRows, kTcNq);
        const uint32_t taps_base = smem_addr(s_taps);
        // Toeplitz form: this warp's block b = r0 of 32 outputs is active for
        // the tile's k-steps [4 b, 4 b + KB / 8); T hi at taps_base, T lo
        // 128 KB bytes on; 8-column groups 32 KB bytes apart
        const int KB = tc_KB(H);
        const int s_lo = 4 * r0, s_hi = s_lo + KB / 8;
        const uint32_t t_sbo = 32u * (uint32_t)KB;
        const uint32_t t_lo = taps_base + 128u * (uint32_t)KB;
        if constexpr (TOEP) {
            const int kb_first = s_lo / (kTcKB / 8), kb_last = (s_hi - 1) / (kTcKB / 8);
            const uint32_t d = tmem + (uint32_t)(r0 * kTcNq);  // block r0 of the accumulator
            unsigned g = 0;
            for (unsigned i = 0; i < n_tiles; ++i) {
                for (int kb = 0; kb < n_kb; ++kb, ++g) {
                    const int t = (int)(g % (unsigned)nA);
                    if (!wait(&a_full[t], (g / (unsigned)nA) & 1u)) goto done;
                    // the epilogue must have read this block of the previous tile
                    if (kb == kb_first && i >= 1 && !wait(&acc_empty[r0], (i - 1) & 1u))
                        goto done;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    if (lane == 0) {
                        const uint32_t a_hi = tmem + acol0 + (uint32_t)t * kTcACols;
#pragma unroll
                        for (int ks = 0; ks < kTcKB / 8; ++ks) {
                            const int st = kb * (kTcKB / 8) + ks;  // k-step of the tile
                            if (st >= s_lo && st < s_hi) {
                                const uint32_t ah = a_hi + (uint32_t)(8 * ks);
                                const uint32_t al = ah + (uint32_t)kTcKB;
                                // rows u' = 8 st - 32 b .. + 7 of T: (u' / 4) x 128 bytes
                                const uint32_t off = 32u * (uint32_t)(8 * st - 32 * r0);
                                const uint64_t dbh = smem_desc(taps_base + off, 128, t_sbo);
                                const uint64_t dbl = smem_desc(t_lo + off, 128, t_sbo);
                                tc_mma_ts(d, ah, dbh, idesc, st > s_lo ? 1u : 0u);
                                tc_mma_ts(d, ah, dbl, idesc, 1u);
                                tc_mma_ts(d, al, dbh, idesc, 1u);
                            }
                        }
                        tc_commit(&a_empty[t]);                      // A stage t may be refilled
                        if (kb == kb_last) tc_commit(&acc_full[r0]);  // the block is complete
                    }
                    __syncwarp();
                }
            }
        } else {
            unsigned g = 0;
            for (unsigned i = 0; i < n_tiles; ++i) {
                const int a = (int)(i & 1u);
                // the epilogue must have drained this accumulator (tile i - 2)
                if (i >= 2 && !wait(&acc_empty[a], ((i >> 1) - 1) & 1u)) goto done;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dacc = tmem + (uint32_t)a * kTcAccCols;
                for (int kb = 0; kb < n_kb; ++kb, ++g) {
                    const int t = (int)(g % (unsigned)kTcAStages);
                    if (!wait(&a_full[t], (g / (unsigned)kTcAStages) & 1u)) goto done;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    if (lane == 0) {
                        const int u0 = kb * kTcKB;
                        const int nks = min(kTcKB, K - u0) / 8;
                        // A: 8 TMEM columns per k-step (hi, then lo 64 columns on);
                        // B: the phase's tap array, 8 samples (32 B) per k-step, in
                        // 16-byte descriptor units
                        const uint32_t a_hi = tmem + kTcACol0 + (uint32_t)t * kTcACols;
                        uint64_t dbh0[kTcPhasesPerWarp], dbl0[kTcPhasesPerWarp];
#pragma unroll
                        for (int rr = 0; rr < kTcPhasesPerWarp; ++rr) {
                            const int r = r0 + rr;
                            dbh0[rr] = smem_desc(taps_base + (uint32_t)(r * Z * 4 + u0 * 4), 16, 128);
                            dbl0[rr] = smem_desc(taps_base + (uint32_t)((4 + r) * Z * 4 + u0 * 4), 16, 128);
                        }
                        const uint32_t acc0 = kb > 0 ? 1u : 0u;
#pragma unroll
                        for (int ks = 0; ks < kTcKB / 8; ++ks) {
                            if (ks < nks) {
                                const uint32_t ah = a_hi + (uint32_t)(8 * ks);
                                const uint32_t al = ah + (uint32_t)kTcKB;
#pragma unroll
                                for (int rr = 0; rr < kTcPhasesPerWarp; ++rr) {
                                    const uint32_t d = dacc + (uint32_t)((r0 + rr) * kTcNq);
                                    const uint64_t dbh = dbh0[rr] + (uint64_t)(2 * ks);
                                    const uint64_t dbl = dbl0[rr] + (uint64_t)(2 * ks);
                                    tc_mma_ts(d, ah, dbh, idesc, (ks > 0) ? 1u : acc0);
                                    tc_mma_ts(d, ah, dbl, idesc, 1u);
                                    tc_mma_ts(d, al, dbh, idesc, 1u);
                                }
                            }
                        }
                        tc_commit(&a_empty[t]);                    // A stage t may be refilled
                        if (kb == n_kb - 1) tc_commit(&acc_full[a]);  // the tile is complete
                    }
                    __syncwarp();
                }
            }
        }
    } else if (warp >= 4 && warp < 8) {
        // ------------------------------ epilogue -----------------------------
        const int m = (warp & 3) * 32 + lane;  // TMEM lane = row of the tile
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        for (unsigned i = 0; TOEP && i < n_tiles; ++i) {
            // Toeplitz form: block b (accumulator columns 32 b..) holds outputs
            // t0 + 32 b ..; it is read, handed back to its MMA warp, then stored
            const TcTile tl = tc_tile(p, blockIdx.x + i * gridDim.x);
            const EnvTcJob &jb = *tl.job;
            const bool vec = (jb.T & 3) == 0;
            const bool vec8 = (jb.T & 7) == 0 && (reinterpret_cast<uintptr_t>(jb.img) & 31) == 0;
            const int row = tl.row0 + m;
            const bool row_ok = row < jb.M;
            float *irow = jb.img + (size_t)(row_ok ? row : 0) * jb.T;
#pragma unroll 1
            for (int b = 0; b < kTcMmaWarps; ++b) {
                // every epilogue thread takes the same branch (named barriers follow)
                if (!epi_all(wait(&acc_full[b], i & 1u))) goto done;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float v[2][16];
                tmem_ld16(lane_base + (uint32_t)(b * kTcNq), v[0]);
                tmem_ld16(lane_base + (uint32_t)(b * kTcNq + 16), v[1]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&acc_empty[b]);
                const int tq = tl.t0 + b * kTcNq;
                if (jb.use_tma_store) {
                    // row m's 32 outputs into store buffer (4 i + b) & 1 at the
                    // 128-byte swizzled chunk positions, then one tensor store of
                    // the 32 x 128 box (rows past M and outputs past T clipped)
                    unsigned char *ob = obuf + (size_t)((4 * i + b) & 1u) * kTcOutBytes;
                    if (m == 0) bulk_wait_read<1>();  // the store two blocks back has read it
                    epi_sync();
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        *reinterpret_cast<float4 *>(ob + m * 128 + (((c & 7) ^ (m & 7)) << 4)) =
                            make_float4(v[c >> 2][4 * (c & 3)], v[c >> 2][4 * (c & 3) + 1],
                                        v[c >> 2][4 * (c & 3) + 2], v[c >> 2][4 * (c & 3) + 3]);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    epi_sync();
                    if (m == 0) {
                        tma_store_2d(&jb.omap, ob, tq, tl.row0);
                        bulk_commit();
                    }
                } else if (row_ok && vec8 && tq + kTcNq <= jb.T) {
#pragma unroll
                    for (int r = 0; r < 2; ++r)
#pragma unroll
                        for (int k = 0; k < 16; k += 8)
                            st_global_v8(irow + tq + 16 * r + k, v[r][k], v[r][k + 1],
                                         v[r][k + 2], v[r][k + 3], v[r][k + 4], v[r][k + 5],
                                         v[r][k + 6], v[r][k + 7]);
                } else if (row_ok) {
#pragma unroll
                    for (int r = 0; r < 2; ++r)
#pragma unroll
                        for (int k = 0; k < 16; k += 4) {
                            const int t = tq + 16 * r + k;
                            if (vec && t + 3 < jb.T) {
                                *reinterpret_cast<float4 *>(irow + t) =
                                    make_float4(v[r][k], v[r][k + 1], v[r][k + 2], v[r][k + 3]);
                            } else {
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (t + e < jb.T) irow[t + e] = v[r][k + e];
                            }
                        }
                }
            }
        }
        for (unsigned i = 0; !TOEP && i < n_tiles; ++i) {
            const int a = (int)(i & 1u);
            const TcTile tl = tc_tile(p, blockIdx.x + i * gridDim.x);
            const EnvTcJob &jb = *tl.job;
            const bool vec = (jb.T & 3) == 0;
            const bool vec8 = (jb.T & 7) == 0 && (reinterpret_cast<uintptr_t>(jb.img) & 31) == 0;
            if (!wait(&acc_full[a], (i >> 1) & 1u)) goto done;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = tl.row0 + m;
            const bool row_ok = row < jb.M;
            float *irow = jb.img + (size_t)(row_ok ? row : 0) * jb.T;
#pragma unroll 1
            for (int qc = 0; qc < kTcNq; qc += 16) {
                float v[4][16];
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    tmem_ld16(lane_base + (uint32_t)a * kTcAccCols + (uint32_t)(r * kTcNq + qc), v[r]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row_ok && vec8 && tl.t0 + 4 * (kTcNq - qc) <= jb.T) {
                    // the 64 outputs are whole: 8 aligned sectors, columns k + 1 and k
                    // holding outputs t .. t + 7
#pragma unroll
                    for (int k = 0; k < 16; k += 2) {
                        const int t = tl.t0 + 4 * (kTcNq - 2 - qc - k);
                        st_global_v8(irow + t, v[0][k + 1], v[1][k + 1], v[2][k + 1], v[3][k + 1],
                                     v[0][k], v[1][k], v[2][k], v[3][k]);
                    }
                } else if (row_ok) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        // column qc + k of phase r holds output j = 4 (Nq - 1 - qc - k) + r
                        const int t = tl.t0 + 4 * (kTcNq - 1 - qc - k);
                        if (vec && t + 3 < jb.T) {
                            *reinterpret_cast<float4 *>(irow + t) =
                                make_float4(v[0][k], v[1][k], v[2][k], v[3][k]);
                        } else {
#pragma unroll
                            for (int r = 0; r < 4; ++r)
                                if (t + r < jb.T) irow[t + r] = v[r][k];
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&acc_empty[a]);
        }
    }
done:
    // on an abort, give MMAs and copies in flight time to land before the
    // shared memory and TMEM are released
    if (abort_flag) {
        const unsigned long long t0 = global_ns();
        while (global_ns() - t0 < 100000000ull) {
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (TOEP && warp == 4 && lane == 0) bulk_wait_all();  // tensor stores in flight
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 9)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                     : "memory");
}

}  // namespace dmas
