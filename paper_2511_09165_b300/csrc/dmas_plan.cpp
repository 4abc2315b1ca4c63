// Host side of plan creation: validation, the FP64 delay look-up table
// (Sec. II of the DMAS paper: the delays are computed once and kept in a
// delay-matrix look-up table), grouping of neighbouring directions into CTA
// rows, the staged-window geometry of the beamform kernel, and the envelope
// taps.
//
// Compiled with -ffp-contract=off: the delay table must come out bit-identical
// to any other FP64 evaluation in the same operation order (x, then y, then z
// of the projection; centroid as the running sum divided by N).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "dmas_internal.h"

namespace dmas {
namespace {

bool finite(double v) { return std::isfinite(v); }

int floor_to(int v, int a) {  // largest multiple of a that is <= v (v may be < 0)
    int q = v / a;
    if (q * a > v) --q;
    return q * a;
}

long long round_up(long long v, int a) { return ((v + a - 1) / a) * a; }

// Hilbert-curve index of (x, y) on a 2^bits x 2^bits grid.  Each level picks
// the quadrant, adds its index times the quadrant's cell count, then rotates or
// reflects the coordinates so the sub-curve has the standard orientation.
uint64_t hilbert_index(uint32_t x, uint32_t y, int bits) {
    uint64_t d = 0;
    for (uint32_t s = 1u << (bits - 1); s > 0; s >>= 1) {
        uint32_t rx = (x & s) ? 1u : 0u;
        uint32_t ry = (y & s) ? 1u : 0u;
        d += (uint64_t)s * (uint64_t)s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = s - 1 - (x & (s - 1));
                y = s - 1 - (y & (s - 1));
            }
            std::swap(x, y);
        }
        x &= (s - 1);
        y &= (s - 1);
    }
    return d;
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations; columns of V
// are eigenvectors, w the eigenvalues.
void jacobi3(double A[3][3], double V[3][3], double w[3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        if (off < 1e-30) break;
        for (int p = 0; p < 2; ++p) {
            for (int q = p + 1; q < 3; ++q) {
                if (std::fabs(A[p][q]) < 1e-300) continue;
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) /
                           (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < 3; ++k) {  // A <- A J
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = cs * akp - sn * akq;
                    A[k][q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < 3; ++k) {  // A <- J^T A
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = cs * apk - sn * aqk;
                    A[q][k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < 3; ++k) {  // V <- V J
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = cs * vkp - sn * vkq;
                    V[k][q] = sn * vkp + cs * vkq;
                }
            }
        }
    }
    for (int i = 0; i < 3; ++i) w[i] = A[i][i];
}

// Order directions so that runs of kGroup consecutive entries have similar
// delay vectors.  Delays are linear in u through the centred array positions,
// so u is projected on the array's two principal axes and sorted along a
// Hilbert curve over that plane (exact for planar arrays).
std::vector<int> direction_order(const std::vector<double> &xyz, int N,
                                 const std::vector<double> &u, int M) {
    std::vector<int> order(M);
    std::iota(order.begin(), order.end(), 0);
    if (M <= kGroup) return order;
    double cen[3] = {0, 0, 0};
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) cen[a] += xyz[3 * i + a];
    for (int a = 0; a < 3; ++a) cen[a] /= N;
    double C[3][3] = {{0}};
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                C[a][b] += (xyz[3 * i + a] - cen[a]) * (xyz[3 * i + b] - cen[b]);
    double V[3][3], w[3];
    jacobi3(C, V, w);
    int idx[3] = {0, 1, 2};
    std::sort(idx, idx + 3, [&](int a, int b) { return w[a] > w[b]; });
    double e1[3], e2[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = V[a][idx[0]] * std::sqrt(std::max(w[idx[0]], 0.0));
        e2[a] = V[a][idx[1]] * std::sqrt(std::max(w[idx[1]], 0.0));
    }
    std::vector<double> px(M), py(M);
    double lo = 1e300, hi = -1e300;
    for (int k = 0; k < M; ++k) {
        px[k] = u[3 * k] * e1[0] + u[3 * k + 1] * e1[1] + u[3 * k + 2] * e1[2];
        py[k] = u[3 * k] * e2[0] + u[3 * k + 1] * e2[1] + u[3 * k + 2] * e2[2];
        lo = std::min(lo, std::min(px[k], py[k]));
        hi = std::max(hi, std::max(px[k], py[k]));
    }
    const int bits = 16;
    double scale = (hi > lo) ? ((1u << bits) - 1) / (hi - lo) : 0.0;
    std::vector<uint64_t> key(M);
    for (int k = 0; k < M; ++k) {
        uint32_t qx = (uint32_t)std::lround((px[k] - lo) * scale);
        uint32_t qy = (uint32_t)std::lround((py[k] - lo) * scale);
        key[k] = hilbert_index(qx, qy, bits);
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return key[a] < key[b]; });
    return order;
}

}  // namespace

dmas_status build_host_plan(const dmas_plan_desc &d, HostPlan &hp, std::string *why) {
    auto fail = [&](const char *msg) {
        if (why) *why = msg;
        return DMAS_EINVAL;
    };
    if (d.n_mics < 1 || d.n_mics > 4096) return fail("n_mics must be in 1..4096");
    if (d.n_dirs < 1 || d.n_dirs > (1 << 20)) return fail("n_dirs must be in 1..2^20");
    if (d.n_samples < 1 || d.n_samples > (1 << 24)) return fail("n_samples must be in 1..2^24");
    if (d.order < 1 || d.order > 8) return fail("order must be in 1..8");
    if (!finite(d.fs) || d.fs <= 0.0) return fail("fs must be finite and > 0");
    if (d.delay_mode != DMAS_DELAY_ROUND && d.delay_mode != DMAS_DELAY_LINEAR)
        return fail("unknown delay_mode");
    if (d.chan_prec < DMAS_CH_F32 || d.chan_prec > DMAS_CH_BF16) return fail("unknown chan_prec");
    if (d.ng_prec != DMAS_NG_CF32 && d.ng_prec != DMAS_NG_F64 && d.ng_prec != DMAS_NG_F32)
        return fail("unknown ng_prec");
    if (d.flags & ~(DMAS_F_CF | DMAS_F_ENVELOPE)) return fail("unknown flag bits");
    if (!finite(d.cf_eps)) return fail("cf_eps must be finite");
    if (d.mf_len < 0 || d.mf_len > kMfMaxLen || (d.mf_len > 0) != (d.mf_signal != nullptr))
        return fail("mf_signal and mf_len: both absent, or 1..8192 samples");
    hp.mf.clear();
    for (int k = 0; k < d.mf_len; ++k) {
        if (!std::isfinite(d.mf_signal[k])) return fail("mf_signal holds a non-finite value");
        hp.mf.push_back(d.mf_signal[k]);
    }
    if ((double)d.n_dirs * (double)d.n_samples > 17179869184.0)
        return fail("n_dirs * n_samples exceeds 2^34");

    const int N = d.n_mics, M = d.n_dirs, T = d.n_samples;
    hp.N = N; hp.M = M; hp.T = T; hp.order = d.order;
    hp.delay_mode = d.delay_mode; hp.flags = d.flags;
    hp.chan_prec = d.chan_prec; hp.ng_prec = d.ng_prec;
    hp.fs = d.fs; hp.c = d.c;
    hp.cf_eps = d.cf_eps > 0.0 ? d.cf_eps : 1e-30;
    if ((float)hp.cf_eps <= 0.0f) return fail("cf_eps underflows in float32");

    // ---- delay table tau[M][N] in FP64 ----------------------------------
    std::vector<double> tau((size_t)M * N);
    std::vector<double> xyz, u;
    const bool geometric = (d.delays_s == nullptr);
    if (!geometric) {
        for (size_t k = 0; k < (size_t)M * N; ++k) {
            if (!finite(d.delays_s[k])) return fail("delays_s holds a non-finite value");
            tau[k] = d.delays_s[k];
        }
    } else {
        if (!d.mic_xyz) return fail("mic_xyz is required without delays_s");
        if (!d.dir_unit && !d.dir_azel) return fail("dir_unit or dir_azel is required");
        if (!finite(d.c) || d.c <= 0.0) return fail("c must be finite and > 0");
        xyz.assign(d.mic_xyz, d.mic_xyz + 3 * (size_t)N);
        for (double v : xyz)
            if (!finite(v)) return fail("mic_xyz holds a non-finite value");
        u.resize(3 * (size_t)M);
        if (d.dir_unit) {
            for (size_t k = 0; k < 3 * (size_t)M; ++k) u[k] = d.dir_unit[k];
        } else {
            for (int k = 0; k < M; ++k) {
                double th = d.dir_azel[2 * k], ph = d.dir_azel[2 * k + 1];
                u[3 * k + 0] = std::sin(th) * std::cos(ph);
                u[3 * k + 1] = std::sin(ph);
                u[3 * k + 2] = std::cos(th) * std::cos(ph);
            }
        }
        for (double v : u)
            if (!finite(v)) return fail("direction holds a non-finite value");
        double cx = 0.0, cy = 0.0, cz = 0.0;
        for (int i = 0; i < N; ++i) {
            cx += xyz[3 * i + 0];
            cy += xyz[3 * i + 1];
            cz += xyz[3 * i + 2];
        }
        cx /= (double)N;
        cy /= (double)N;
        cz /= (double)N;
        for (int k = 0; k < M; ++k) {
            for (int i = 0; i < N; ++i) {
                double dx = xyz[3 * i + 0] - cx;
                double dy = xyz[3 * i + 1] - cy;
                double dz = xyz[3 * i + 2] - cz;
                double proj = dx * u[3 * k + 0];
                proj = proj + dy * u[3 * k + 1];
                proj = proj + dz * u[3 * k + 2];
                tau[(size_t)k * N + i] = -proj / d.c;
            }
        }
    }
    hp.shift.resize((size_t)M * N);
    hp.frac.resize((size_t)M * N);
    const double kMaxShift = 4194304.0;  // 2^22 samples
    for (size_t k = 0; k < (size_t)M * N; ++k) {
        double delta = tau[k] * d.fs;
        if (!(std::fabs(delta) <= kMaxShift)) return fail("a delay exceeds 2^22 samples");
        if (d.delay_mode == DMAS_DELAY_ROUND) {
            hp.shift[k] = (int32_t)std::llround(delta);
            hp.frac[k] = 0.0f;
        } else {
            double j = std::floor(delta);
            hp.shift[k] = (int32_t)j;
            hp.frac[k] = (float)(delta - j);
        }
    }

    // ---- direction groups -----------------------------------------------
    std::vector<int> order;
    if (geometric) {
        order = direction_order(xyz, N, u, M);
    } else {
        order.resize(M);
        std::iota(order.begin(), order.end(), 0);
    }
    const int G = (M + kGroup - 1) / kGroup;
    hp.n_groups = G;
    hp.gdir.assign((size_t)G * kGroup, -1);
    for (int k = 0; k < M; ++k) hp.gdir[k] = order[k];
    hp.gws.assign((size_t)G * N, 0);
    hp.rel.assign((size_t)G * N * kGroup, 0);
    hp.gfrac.assign((size_t)G * N * kGroup, 0.0f);
    const int lin = (d.delay_mode == DMAS_DELAY_LINEAR) ? 1 : 0;
    long long spread = 0;
    int ws_min = 0, ws_max = 0;
    bool first = true;
    for (int g = 0; g < G; ++g) {
        for (int i = 0; i < N; ++i) {
            int dmin = 0, dmax = 0;
            bool any = false;
            for (int s = 0; s < kGroup; ++s) {
                int dir = hp.gdir[(size_t)g * kGroup + s];
                if (dir < 0) continue;
                int sh = hp.shift[(size_t)dir * N + i];
                if (!any) { dmin = dmax = sh; any = true; }
                dmin = std::min(dmin, sh);
                dmax = std::max(dmax, sh);
            }
            int ws = floor_to(dmin, kAlign);
            hp.gws[(size_t)g * N + i] = ws;
            spread = std::max<long long>(spread, (long long)dmax + lin - ws);
            if (first) { ws_min = ws_max = ws; first = false; }
            ws_min = std::min(ws_min, ws);
            ws_max = std::max(ws_max, ws);
            for (int s = 0; s < kGroup; ++s) {
                int dir = hp.gdir[(size_t)g * kGroup + s];
                size_t o = ((size_t)g * N + i) * kGroup + s;
                if (dir < 0) continue;
                hp.rel[o] = hp.shift[(size_t)dir * N + i] - ws;
                hp.gfrac[o] = hp.frac[(size_t)dir * N + i];
            }
        }
    }
    const size_t eb = chan_elem_bytes(d.chan_prec);
    if (uses_pair_kernel(d.chan_prec, d.order)) {
        // pixel pairs per lane (time tile 64 x pairs): nearest-sample frames
        // with enough work items, and at least one wide tile long, take the
        // wide tile
        const int rp = round_pairs(d.order);
        const size_t wide_items = (size_t)G * (size_t)((T + 64 * rp - 1) / (64 * rp));
        hp.pairs = lin ? kLinPairs : (wide_items >= kWideMinItems && T >= 64 * rp ? rp : 2);
        hp.tile = 64 * hp.pairs;
    } else {
        hp.pairs = 0;
        hp.tile = kTimeTile;
    }
    long long window = round_up(hp.tile + spread, kAlign);
    // The persistent pair kernel (nearest-sample delays) double-buffers its
    // staged windows; the interpolated-delay pair kernel stages a root and a
    // raw-sample window per microphone.
    const bool pair = uses_pair_kernel(d.chan_prec, d.order);
    const bool persistent = pair && !lin;
    const size_t budget = persistent ? kPairSmemBudget - 2 * 256
                                     : kWindowSmemBudget - (pair ? 8 * 6 * 32 * 4 : 0);
    const size_t tab = (size_t)kGroup * 4 * (lin ? 2 : 1);
    auto bytes_per_mic = [&](long long w) {
        return persistent ? 2 * ((size_t)w * eb + tab)
                          : (pair ? lin_mic_bytes((int)w) + (size_t)kGroup * 12
                                  : (size_t)w * eb + tab);
    };
    if (persistent && hp.pairs > 2 && bytes_per_mic(window) > budget) {
        // a delay spread too wide for the wide tile: back to two pairs
        hp.pairs = 2;
        hp.tile = 64 * hp.pairs;
        window = round_up(hp.tile + spread, kAlign);
    }
    const size_t per_mic = bytes_per_mic(window);
    if (per_mic > budget)
        return fail("a direction group's delay spread does not fit in shared memory");
    hp.window = (int)window;
    hp.mic_chunk = (int)std::min<size_t>((size_t)N, budget / per_mic);
    if (persistent) {  // balanced chunks
        const int n_chunks = (N + hp.mic_chunk - 1) / hp.mic_chunk;
        hp.mic_chunk = (N + n_chunks - 1) / n_chunks;
    }
    if (pair && lin) {
        const size_t mb = lin_mic_bytes(hp.window);
        hp.gsel.assign(hp.rel.size(), 0);
        hp.gwf2.assign(hp.rel.size() * 2, 0.0f);
        for (int g = 0; g < G; ++g)
            for (int i = 0; i < N; ++i)
                for (int s = 0; s < kGroup; ++s) {
                    const size_t o = ((size_t)g * N + i) * kGroup + s;
                    const int off = hp.rel[o];
                    const size_t blk = (size_t)(i % hp.mic_chunk) * mb;
                    hp.gsel[o] = (int32_t)(blk + (size_t)off * 4);
                    const float f = hp.gfrac[o];
                    hp.gwf2[o * 2 + 0] = f;
                    hp.gwf2[o * 2 + 1] = f;
                }
    }
    hp.spread = (int)spread;
    // Every-order pass: 128-sample tiles for nearest-sample delays, 64 for
    // interpolated ones; as many microphones per stage as fit two stages in
    // the budget, in balanced chunks.
    hp.mo_tile = hp.mo_window = hp.mo_chunk = hp.mo_tiles = 0;
    hp.mo_halves = 1;
    const size_t mo_budget = lin ? kOrdersSmemBudget : kOrdersRoundSmemBudget;
    // interpolated delays, every microphone in one stage: a tile of three (or
    // two) 64-sample pieces summed one after the other from one staged window
    // (measured on B300, hemisphere frame: 2.07 ms with one piece per CTA, 1.96
    // with two, 1.94 with three)
    int mo_h = 0;
    for (int hv = 3; pair && lin && hv >= 2 && mo_h == 0; --hv)
        if (orders_smem_bytes(d.order, lin, N,
                              (int)round_up(hv * orders_tile(lin) + spread, kAlign), hv) <=
            mo_budget)
            mo_h = hv;
    if (mo_h > 0) {
        hp.mo_halves = mo_h;
        hp.mo_tile = mo_h * orders_tile(lin);
        hp.mo_window = (int)round_up(hp.mo_tile + spread, kAlign);
        hp.mo_chunk = N;
        hp.mo_tiles = (T + hp.mo_tile - 1) / hp.mo_tile;
    } else if (pair) {
        const int mt = orders_tile(lin);
        const int mw = (int)round_up(mt + spread, kAlign);
        int chunk = 0;
        while (chunk < N && orders_smem_bytes(d.order, lin, chunk + 1, mw) <=
                                   (lin ? kOrdersSmemBudget : kOrdersRoundSmemBudget))
            ++chunk;
        if (chunk > 0) {
            const int n_chunks = (N + chunk - 1) / chunk;
            hp.mo_tile = mt;
            hp.mo_window = mw;
            hp.mo_chunk = (N + n_chunks - 1) / n_chunks;
            hp.mo_tiles = (T + mt - 1) / mt;
        }
    }
    hp.n_tiles = (T + hp.tile - 1) / hp.tile;
    hp.padl = (int)round_up(std::max(0, -ws_min), kAlign);
    long long read_end = (long long)hp.padl + (long long)(hp.n_tiles - 1) * hp.tile +
                         ws_max + window;
    if (hp.mo_chunk > 0)  // the every-order pass's last window as well
        read_end = std::max<long long>(read_end, (long long)hp.padl +
                                                     (long long)(hp.mo_tiles - 1) * hp.mo_tile +
                                                     ws_max + hp.mo_window);
    hp.row = (int)round_up(std::max<long long>(read_end, (long long)hp.padl + T), kAlign);

    // ---- envelope taps (windowed sinc, Hamming, unit DC gain) -----------
    if (d.flags & DMAS_F_ENVELOPE) {
        double fc = d.env_cutoff_hz > 0.0 ? d.env_cutoff_hz : 5000.0;
        if (!finite(fc) || fc >= 0.5 * d.fs) return fail("env_cutoff_hz must be below fs/2");
        long long L = d.env_taps;
        if (L == 0) L = 2 * (long long)std::ceil(d.fs / fc) + 1;
        if (L < 1 || L > kMaxTaps || (L % 2) == 0)
            return fail("envelope length must be odd and at most 1023 taps");
        hp.env_fc = fc;
        hp.L = (int)L;
        const int H = (int)(L - 1) / 2;
        std::vector<double> h(L);
        double sum = 0.0;
        for (int k = -H; k <= H; ++k) {
            double ideal = (k == 0) ? 2.0 * fc / d.fs
                                    : std::sin(2.0 * M_PI * fc * k / d.fs) / (M_PI * k);
            double win = (H == 0) ? 1.0 : 0.54 + 0.46 * std::cos(M_PI * k / H);
            h[k + H] = win * ideal;
            sum += h[k + H];
        }
        hp.taps.resize(L);
        for (int k = 0; k < L; ++k) hp.taps[k] = (float)(h[k] / sum);
    } else {
        hp.L = 0;
    }
    return DMAS_OK;
}

}  // namespace dmas
