// Discrepancy + top-k (Algorithm 1, steps 4-5) on the 5th-generation tensor
// cores, fused so the J x N distance matrix never reaches memory.
//
// d_jn = sum_l w_l (y_jl - x_nl)^2 = ||yh_j||^2 + ||xh_n||^2 - 2 yh_j . xh_n with
// yh = sqrt(w)(y - mu), xh = sqrt(w)(x - mu) (mu = mean voxel TAC; distances
// are translation invariant).  The ranking key d' = ||xh||^2 - 2 yh . xh is one
// GEMM: voxel rows A = [yh .., 1, 1, 1], draw rows B = [-2 xh .., n_hi, n_mid, n_lo]
// where the norm column n is split over three bf16 columns.
//   ABC_FP32:  yh, xh split into bf16 hi + lo; A = [yh_hi, yh_hi, yh_lo, 1,1,1],
//              B = [-2xh_hi, -2xh_lo, -2xh_hi, n_hi, n_mid, n_lo]: three bf16
//              products per term, |error| <= E(voxel) (bound below).
//   split form (ABC_BF16_RESCORE, ABC_SPLIT_DRAWS): A = [yh_bf, yh_bf, 1,1,1],
//              B = [-2xh_hi, -2xh_lo, n_hi, n_mid, n_lo] with n = ||xh||^2 - 2 xh.r
//              (r = xh - xh_hi - xh_lo): two products per term.  The key is then
//              exact up to c0 (a per-voxel constant) and 2 (yh - xh).(r + delta)
//              (delta = the voxel row's rounding), which vanishes with the distance
//              (need_key / dist_ub below).
//
// Kernel `k_tc_topk`: one CTA owns 128 voxels (one TMEM lane each) and streams
// the draw tiles through shared memory (TMA, 128-byte swizzle).  Warp roles:
// 0 = TMA producer, 1 = TMEM allocator + MMA issuer (one thread), 2.. = epilogue
// (thread <-> voxel).  Accumulators are double-buffered in TMEM so the MMA of tile
// t+1 overlaps the epilogue of tile t.  The epilogue reads 32 columns at a time and
// takes their minimum; a thread whose minimum is within its voxel's threshold
// appends each passing (key, draw index) pair to the voxel's candidate list.  When
// a list could overflow, the warp compacts it (radix select of the kt-th key,
// in-place filtering) and tightens the threshold, so a list always holds every draw
// whose key is at most its voxel's threshold.
//
// Pilot passes of the same kernel over every 16th (then 256th, ...) draw (a
// strided TMA tensor map) set each voxel's threshold for the next pass.  The
// coarser levels aim at a rank (about 1.5 kt draws of the next finer level); the
// finest level of the split form instead finds the key of rank rk (the k-th
// distance's upper bound, four standard deviations safe) and k_need_threshold turns
// it into need_key(dist_ub(key)): every draw the certificate below can ask for.
// Nothing relies on the prediction for correctness.
//
// Kernel `k_finalize` (one warp per voxel) re-scores the net exactly as
// sum_l w_l (y_l - x_l)^2 in fp32, selects the exact k-th distance d_k, and
// certifies the result: every draw outside the net has computed key > T_out, so
// none can be within d_k when T_out >= the largest key a draw within d_k can have
// (need_key for the split form; d_k - ||yh||^2 + E for ABC_FP32).  An uncertified
// voxel is resolved by an exact fp32 scan of all draws, which makes every accepted
// set the exact fp32 top-k.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "common.cuh"
#include "select.cuh"
#include "tc_ptx.cuh"

using namespace vpet;

namespace {

constexpr int BM = 128;                       // voxels per CTA tile = TMEM lanes
constexpr int KBLK = 64;                      // bf16 per K-block (128-byte rows)
constexpr int A_KBLK_BYTES = BM * KBLK * 2;   // 16 KB
// Fused kernel: TMA warp, MMA warp, then the epilogue warps: four (one thread per
// voxel and tile: top-r pilots and 64-draw tiles) or eight with 128-draw tiles
// (two per TMEM lane quadrant, each taking every other 32-column chunk of a tile
// and keeping its own half of the voxel's candidate list).
constexpr int tc_epi_warps(bool topr, int bn) { return (topr || bn == 64) ? 4 : 8; }
constexpr int tc_threads(bool topr, int bn) { return 64 + 32 * tc_epi_warps(topr, bn); }
// Per-thread key rows: the top-r variants keep their kept keys there, the one-K-block list
// variants read passing keys back from them (shared memory allows it next to two CTAs per
// SM); the wider list variants pick passing keys from registers instead.
constexpr bool tc_rows(int nkb, bool topr) { return topr || nkb == 1; }

constexpr uint64_t WAIT_NS_DEFAULT = 2000000000ull;   // 2 s bound on any barrier wait
constexpr int MAXL = 64;
constexpr int ORDER_BITS = 10;                 // bits per ordering feature (30-bit Morton key)
constexpr int ORDER_BUCKET_BITS = 18;
constexpr int ORDER_BUCKETS = 1 << ORDER_BUCKET_BITS;   // counting-sort buckets
constexpr int MAX_PILOT_LEVELS = 4;
constexpr int ROW_LD = 36;                     // floats per epilogue thread's key row (16-byte rows, conflict-free)
// A pilot level with a small target rank keeps each voxel's r smallest keys per
// epilogue thread in shared memory (the key rows and compaction histograms,
// unused in that mode): at most this many.
constexpr int TOPR_MAX = (128 * ROW_LD + 4 * 256) / 128;
constexpr int MAX_ITEMS = 64;                 // scans per batched launch
// Work items per rescued voxel tile: the rescue pass usually has few voxel tiles, each of
// which would otherwise stream all its draw tiles through one CTA.
constexpr int RESCUE_SEGMENTS = 8;
// A scan of at most this many voxels may queue all of them for the rescue pass.
constexpr int64_t RESCUE_ALL_VOXELS = 16384;

struct Weights {
    float w[MAXL];
    float sw[MAXL];   // sqrt(w)
};

// Launch choices the autotuner varies (abc_tuning in the C ABI).
struct Tuning {
    int bn;               // draws per tile: 64 or 128
    int ctas_per_sm;      // persistent CTAs per SM (capped by occupancy)
    int pilot_stride;     // draw stride of each pilot level: 8, 16 or 32
    float pilot_factor;   // predicted candidates / net size at the next finer level (>= 1.25)
};

// Built-in defaults (measured on B300): 128-draw tiles, two CTAs per SM with
// eight epilogue warps, for the bf16 and fp32-split operands (brain lp-ntPET
// k = 500: main pass 30.5 ms against 37.5 with three 64-draw CTAs; total-body
// FDG k = 200: step 385 ms against 397); the split-draws operands (two K-blocks)
// keep three 64-draw CTAs per SM, as 128-draw tiles would leave one CTA per SM.
// ABC_FP32 aims its pilots at 2.25 kt candidates: its net (2k) takes the list as
// it stands, whose threshold must clear the certificate's error margin (at 1.5 kt
// ten times more C2 voxels fell back to the exact scan).
Tuning default_tuning(int mode) {
    if (mode == ABC_FP32) return Tuning{128, 2, 8, 2.25f};
    // split form: the finest pilot (every 8th draw) estimates the k-th distance for the
    // main pass's per-voxel threshold; a finer sample needs less rank margin, so lists
    // are shorter and fewer reach their capacity
    return Tuning{128, 2, 8, 1.5f};
}

// The built-in tuning of a single-scan call: 128-draw tiles for every shape (with two K-blocks
// their list variants keep two CTAs per SM by picking passing keys from registers); the fast
// form's finest pilot takes every 16th draw when k >= 400.  The finest pilot's rank rk must
// sit four standard deviations above k / stride, which costs relatively less margin the larger
// k / stride is: for k = 500 stride 16 places the threshold near rank 2.1 k (stride 8: 1.9 k) at
// half the pilot's work (brain volume: 73.3 against 77.2 ms per step), for k = 200 near 3.2 k
// (stride 8: 2.2 k; total body: 231.9 against 222.4 ms).
Tuning default_tuning_for_shape(int mode, int L, int k) {
    (void)L;
    Tuning t = default_tuning(mode);
    if (mode != ABC_FP32 && k >= 400) t.pilot_stride = 16;
    return t;
}

// bf16 columns of the packed operands per frame: products per term of the key.
__host__ __device__ inline int cols_per_frame(int mode) { return mode == ABC_FP32 ? 3 : 2; }

struct Layout {
    int mode;          // ABC_FP32 or ABC_SPLIT_DRAWS (ABC_BF16_RESCORE runs as the latter)
    int L, k, Kp, nkb, C, kt, cap, sortcap;
    int rk;                            // split form: rank of the k-th-distance bound in the finest pilot
    int nlev;                          // pilot levels (finest first)
    int lev_rank[MAX_PILOT_LEVELS];
    int64_t lev_stride[MAX_PILOT_LEVELS];
    int64_t J, N, Jp, Np;
    int npart;
    size_t off_mu, off_part, off_ynorm, off_c0, off_dn, off_a, off_b, off_keys, off_idx, off_cnt, off_thr, off_thr0,
        off_perm, off_feat, off_hist, off_xperm, off_xfeat, off_xhist, off_fy, off_fx, off_tbox, off_ktile,
        off_kcount, off_xs, off_w, off_rq, off_rrow, off_rthr, off_ra, total;
    int64_t rcap;                      // split form: voxels the rescue pass can take (0: none)
    int G;                             // centring groups (split form): packed voxel rows [g Jg, (g+1) Jg)
    int64_t Jg;                        // rows per group, a multiple of 128 (every voxel tile lies in one group)
    int64_t rcapa;                     // rescue positions allocated: rcap plus a padded tile per group
    int64_t lrows;                     // candidate-list rows allocated: max(J, rcapa)
    int Cr;                            // rescue pass: list capacity of a queue position (>= C)
    size_t off_tgroup, off_rq2, off_rtg, off_rcnt, off_rthrh;
    int ldxs;                          // row stride (floats) of the packed fp32 draw copy
    int64_t nt64;                      // 64-draw tiles of the draw operand
    int64_t nvt;                       // 128-voxel tiles
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// kp_min: the packed K width is at least this (a batch pads every scan to its widest).
// list_mult (split form): candidate lists hold list_mult x 12 k entries (1, 2 or 4; the batch
// layout chooses it per scan within a memory budget): fewer voxels whose net outgrows its list.
Layout make_layout(int64_t J, int64_t N, int L, int k, int mode, const Tuning& tu, int kp_min = 0, int list_mult = 1,
                   int groups = 1) {
    Layout s;
    memset(&s, 0, sizeof s);
    s.mode = mode;
    s.L = L;
    s.k = k;
    s.J = J;
    s.N = N;
    const int kcols = cols_per_frame(mode) * L + 3;
    s.Kp = (int)vpet_round_up(kcols, KBLK);
    if (s.Kp < kp_min) s.Kp = kp_min;
    s.nkb = s.Kp / KBLK;
    // kt: the net of the FP32 form and the compaction target of every form (2k).  The
    // split form's lists instead hold every draw below a per-voxel threshold that the
    // finest pilot derives from the certificate's own bound (need_key), up to the
    // capacity C below.
    const int64_t net = 2 * (int64_t)k;
    s.kt = (int)(net < N ? net : N);
    s.cap = s.kt + (s.kt / 4 > 64 ? s.kt / 4 : 64);
    // rank, in the finest pilot sample, of the key whose distance bounds the k-th
    // distance from above unless the sample under-represents the draws below it by
    // more than four standard deviations (split form only)
    s.rk = 0;
    if (mode != ABC_FP32) {
        const double sd = tu.pilot_stride;
        int64_t r = (int64_t)ceil((double)k / sd);
        for (int it = 0; it < 200; ++it) {
            if (1.0 - (double)k / (sd * (double)r) >= 4.0 / sqrt((double)r)) break;
            r = r + r / 8 + 1;
        }
        s.rk = (int)r;
    }
    // Pilot levels: level i uses every stride^i-th draw and a target rank
    // r_i = ceil(f r_{i-1} / stride), r_0 = kt, so that about f r_{i-1} draws of
    // the next finer level fall below its threshold.  For a small r_i the rank
    // statistic is noisy (relative sd ~ 1 / sqrt(r_i)), so r_i grows in steps of 1/8 until an
    // under-prediction is more than ~4 sd away.
    s.nlev = 0;
    int64_t rr = s.kt, stride = 1;
    const double f0 = tu.pilot_factor;
    while (s.nlev < MAX_PILOT_LEVELS) {
        int64_t r_next = (int64_t)ceil(f0 * (double)rr / tu.pilot_stride);
        for (int it = 0; it < 40; ++it) {
            const double f = (double)r_next * tu.pilot_stride / (double)rr;   // predicted count / needed
            if (1.0 - 1.0 / f >= 4.0 / sqrt((double)r_next)) break;
            r_next = r_next + r_next / 8 + 1;
        }
        if (s.nlev == 0 && r_next < s.rk) r_next = s.rk;    // the finest pilot list must hold rank rk
        const int64_t n_next = N / (stride * tu.pilot_stride);
        if (n_next < 8 * r_next || n_next < 512) break;
        stride *= tu.pilot_stride;
        rr = r_next;
        s.lev_rank[s.nlev] = (int)rr;
        s.lev_stride[s.nlev] = stride;
        s.nlev++;
    }
    // list capacity: the FP32 form's net is the list as it stands (~2.25 kt); a split-form
    // list holds its voxel's need-sized net, at most 12 k (the certificate's nets measured on
    // the brain and total-body workloads stay below 12 k; a voxel past it takes the exact scan)
    const int64_t cap_entries = mode == ABC_FP32 ? 3 * (int64_t)s.kt + 256
                                                 : 12 * (int64_t)(list_mult > 1 ? list_mult : 1) * k + 256;
    s.C = (int)vpet_round_up(cap_entries, 32);
    s.sortcap = next_pow2(k + 8);     // k plus a few ties at the k-th distance
    if (s.sortcap < 64) s.sortcap = 64;
    s.Jp = vpet_round_up(J > 0 ? J : 1, BM);
    s.Np = vpet_round_up(N > 0 ? N : 1, 128);
    // centring groups: G contiguous runs of whole voxel tiles in the packed (feature) order
    s.G = mode == ABC_FP32 || groups < 1 ? 1 : groups;
    s.Jg = vpet_round_up(vpet_ceil_div(J > 0 ? J : 1, s.G), BM);
    s.G = (int)vpet_ceil_div(J > 0 ? J : 1, s.Jg);
    {
        const int64_t per_group = vpet_ceil_div(s.Jg, 256);
        const int64_t cap = 1024 / s.G > 1 ? 1024 / s.G : 1;
        s.npart = (int)(per_group < cap ? per_group : cap);
        if (s.npart < 1) s.npart = 1;
    }
    size_t o = 0;
    s.off_mu = o; o = align256(o + (size_t)s.G * MAXL * sizeof(float));
    s.off_part = o; o = align256(o + (size_t)s.G * s.npart * MAXL * sizeof(float));
    s.off_ynorm = o; o = align256(o + (size_t)s.Jp * sizeof(float));
    s.off_c0 = o; o = align256(o + (size_t)s.Jp * sizeof(float));
    s.off_dn = o; o = align256(o + (size_t)s.Jp * sizeof(float));
    s.off_a = o; o = align256(o + (size_t)s.Jp * s.Kp * 2);
    s.off_b = o; o = align256(o + (size_t)s.G * s.Np * s.Kp * 2);   // one packed copy per centring group
    // rescue queue of the split form: a quarter of the voxels (all of them in a small scan;
    // the rest of an unusually bad scan takes the exact scan), plus a padded tile per group
    s.rcap = mode == ABC_FP32 ? 0
                              : (J <= RESCUE_ALL_VOXELS ? s.Jp : vpet_round_up(vpet_ceil_div(J > 0 ? J : 1, 4), BM));
    s.rcapa = s.rcap > 0 ? s.rcap + (int64_t)s.G * BM : 0;
    // candidate lists: J rows of C entries; the rescue pass lays the same space out as rcapa
    // rows of Cr entries (the first pass's lists are dead by then), so a queued voxel's net
    // may be several times the first pass's capacity
    s.lrows = J > s.rcapa ? J : s.rcapa;
    s.Cr = s.rcapa > 0 ? (int)((s.lrows * (int64_t)s.C / s.rcapa) & ~(int64_t)1) : 0;
    s.off_keys = o; o = align256(o + (size_t)s.lrows * s.C * sizeof(float));
    s.off_idx = o; o = align256(o + (size_t)s.lrows * s.C * sizeof(int32_t));
    s.off_cnt = o; o = align256(o + (size_t)2 * s.Jp * sizeof(int32_t));     // two half-lists per voxel
    s.off_thr = o; o = align256(o + (size_t)2 * s.Jp * sizeof(float));
    s.off_thr0 = o; o = align256(o + (size_t)s.Jp * sizeof(float));
    s.off_perm = o; o = align256(o + (size_t)s.Jp * sizeof(int32_t));
    s.off_feat = o; o = align256(o + (size_t)3 * s.Jp * sizeof(float) + 8 * sizeof(uint32_t));
    s.off_hist = o; o = align256(o + (size_t)(ORDER_BUCKETS + ORDER_BUCKETS / 1024) * sizeof(uint32_t));
    s.nt64 = s.Np / 64;
    s.nvt = s.Jp / BM;
    s.off_xperm = o; o = align256(o + (size_t)s.Np * sizeof(int32_t));
    s.off_xfeat = o; o = align256(o + (size_t)3 * s.Np * sizeof(float) + 8 * sizeof(uint32_t));
    s.off_xhist = o; o = align256(o + (size_t)(ORDER_BUCKETS + ORDER_BUCKETS / 1024) * sizeof(uint32_t));
    s.off_fy = o; o = align256(o + (size_t)3 * s.Jp * sizeof(float));
    s.off_fx = o; o = align256(o + (size_t)3 * s.Np * sizeof(float));
    s.off_tbox = o; o = align256(o + (size_t)6 * s.nt64 * sizeof(float));
    s.off_ktile = o; o = align256(o + (size_t)s.nvt * s.nt64 * sizeof(int32_t));
    s.off_kcount = o; o = align256(o + (size_t)s.nvt * sizeof(int32_t));
    s.ldxs = (int)vpet_round_up(L, 4);
    s.off_xs = o; o = align256(o + (size_t)s.Np * s.ldxs * sizeof(float));
    s.off_w = o; o = align256(o + MAXL * sizeof(float));
    s.off_tgroup = o; o = align256(o + (size_t)s.nvt * sizeof(int32_t));
    // queue words: count, queued positions in use, then per group its count, cursor and first position,
    // then the rescue lists' capacity
    s.off_rq = o; o = align256(o + (size_t)(2 + 3 * s.G + 2) * sizeof(int32_t));
    s.off_rrow = o; o = align256(o + (size_t)s.rcapa * sizeof(int32_t));
    s.off_rthr = o; o = align256(o + (size_t)s.rcapa * 2 * sizeof(float));   // thresholds, then first-net d_k
    s.off_rq2 = o; o = align256(o + (size_t)s.rcapa * 3 * sizeof(int32_t));   // the queue sorted by group
    s.off_rtg = o; o = align256(o + (size_t)(s.rcapa / BM + 1) * sizeof(int32_t));
    s.off_rcnt = o; o = align256(o + (size_t)2 * s.rcapa * sizeof(int32_t));   // rescue lists: counts, per half
    s.off_rthrh = o; o = align256(o + (size_t)2 * s.rcapa * sizeof(float));    // and final thresholds
    s.off_ra = o; o = align256(o + (size_t)s.rcapa * s.Kp * 2);
    s.total = o;
    return s;
}

// ------------------------------------------------------------------ split-form key bounds
// The split form's key of voxel row a (yh, fp32) and draw row b (xh, fp32): the voxel row
// rounded once to bf16, a' = a + da; the draw row as bf16 hi + lo with residual
// r = b - hi - lo (|r_l| <= 2^-16 |b_l|); the draw's norm column N = ||b||^2 - 2 b.r.
// The MMA computes key = N - 2 a'.(hi + lo), which is exactly
//   key = ||a - b||^2 - ||a||^2 + c0 + 2 (a - b).(r + da) + 2 da.r      (c0 = -2 da.a)
// plus its fp32 accumulation.  The variable part is at most 2 ||a - b|| (||r|| + ||da||):
// it scales with the square root of the distance, so nearby draws are ranked almost
// exactly.  need_key and dist_ub turn that into two bounds, used by the certificate,
// the per-voxel pilot threshold and the tile bound.
struct SplitCoef {
    float cacc;    // fp32 accumulation of the MMA over Kp columns and the split norm: (3 Kp + L + 16) 2^-24
    float slack;   // fp32 sums of the re-score and of ||yh||^2: 4 L 2^-24
};

// The largest computed key a draw can have if its distance to the voxel (as the exact
// fp32 re-score computes it) is at most D.  yn = ||yh||^2, c0, dn = ||da|| of the voxel row.
__host__ __device__ __forceinline__ float need_key(float D, float yn, float c0, float dn, const SplitCoef& c) {
    const float ry = sqrtf(fmaxf(yn, 0.0f));
    const float s = sqrtf(fmaxf(D, 0.0f) * (1.0f + c.slack)) * (1.0f + 0x1p-20f);   // bounds the real distance's root
    const float sp = s + 0x1p-21f * (2.0f * ry + s);       // ||a - b||: fp32 centring and scaling of both rows
    const float R = ry + sp;                                 // >= ||b||
    const float e1 = dn * (1.0f + 0x1p-10f) + 0x1p-16f * R;   // >= ||da|| + ||r||
    const float t = sp * sp - yn * (1.0f - c.slack) + c0 + 2.0f * sp * e1 + 0x1p-15f * dn * (ry + R) +
                    c.cacc * (2.0f * ry * R + R * R);
    return t + 0x1p-20f * (yn + sp * sp + fabsf(c0));
}

// An upper bound on the exact distance of any draw whose computed key is at most T:
// key >= q^2 - ||a||^2 + c0 - 2 q e1 - (rest) with q = ||a - b||, solved for q.
__host__ __device__ __forceinline__ float dist_ub(float T, float yn, float c0, float dn, const SplitCoef& c) {
    if (!(T < 1.0e30f)) return 3.0e38f;
    const float ry = sqrtf(fmaxf(yn, 0.0f));
    const float dnp = dn * (1.0f + 0x1p-10f);
    const float A = 1.0f - 0x1p-15f - c.cacc;
    const float B = 2.0f * dnp + 0x1p-15f * (ry + dn) + 4.0f * c.cacc * ry;
    const float C = T + yn * (1.0f + c.slack) - c0 + 0x1p-14f * dn * ry + 3.0f * c.cacc * yn +
                    0x1p-20f * (yn + fabsf(T) + fabsf(c0));
    const float disc = B * B + 4.0f * A * C;
    if (!(disc >= 0.0f)) return 0.0f;                        // no draw has such a key
    const float q = fmaxf((B + sqrtf(disc)) / (2.0f * A), 0.0f);
    const float sq = q + 0x1p-21f * (2.0f * ry + q);         // back to the exact rows
    return sq * sq * (1.0f + c.slack) * (1.0f + 0x1p-20f);
}

// ------------------------------------------------------------------ packing
// Centring groups.  The key's error scales with the norms of the centred rows, so a
// voxel far from the centre (a small-signal voxel in a scan of large ones) needs a long
// net.  Voxels are processed in a feature order (below), and G contiguous runs of whole
// 128-voxel tiles of that order are each centred on their own mean TAC; the draw operand
// is packed once per group (copies stacked in B), and a work item reads the copy of its
// voxel tile's group.  Distances are translation invariant, so results do not change.

// Column sums of each group's voxels (packed row j is voxel perm[j]; perm null: voxel j),
// npart partial sums per group, then their fp64 total: a deterministic reduction.
__global__ void k_colmean_part(const float* __restrict__ y, int64_t J, int ldy, int L, float* __restrict__ part,
                               int npart, const int32_t* __restrict__ perm, int64_t Jg) {
    __shared__ float red[4][MAXL];
    const int l = threadIdx.x & 63, g = threadIdx.x >> 6;
    const int grp = blockIdx.x / npart, pp = blockIdx.x % npart;
    const int64_t r0 = (int64_t)grp * Jg, r1 = r0 + Jg < J ? r0 + Jg : J;
    const int64_t per = (r1 - r0 + npart - 1) / npart;
    const int64_t j0 = r0 + pp * per, j1 = j0 + per < r1 ? j0 + per : r1;
    float s = 0.0f;
    if (l < L)
        for (int64_t j = j0 + g; j < j1; j += 4) s += y[(perm ? (int64_t)perm[j] : j) * ldy + l];
    red[g][l] = s;
    __syncthreads();
    if (g == 0) part[(size_t)blockIdx.x * MAXL + l] = red[0][l] + red[1][l] + red[2][l] + red[3][l];
}

// mu[g] = group g's column means (one block per group); wdev = the frame weights, kept on
// the device for the finalize
__global__ void k_colmean_final(const float* __restrict__ part, int npart, int64_t J, int64_t Jg,
                                float* __restrict__ mu, Weights W, float* __restrict__ wdev) {
    const int l = threadIdx.x, grp = blockIdx.x;
    double s = 0.0;
    for (int b = 0; b < npart; ++b) s += part[((size_t)grp * npart + b) * MAXL + l];
    const int64_t r0 = (int64_t)grp * Jg, r1 = r0 + Jg < J ? r0 + Jg : J;
    mu[(size_t)grp * MAXL + l] = (float)(s / (double)(r1 - r0));
    if (grp == 0) wdev[l] = W.w[l];
}

// tgroup[t] = the centring group of voxel tile t
__global__ void k_tile_groups(int32_t* __restrict__ tgroup, int64_t nvt, int64_t Jg) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nvt) tgroup[t] = (int32_t)(t * BM / Jg);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ __nv_bfloat16 bf(float v) { return __float2bfloat16_rn(v); }
// Two values rounded to bf16, a in the low half (the lower address)
__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(bf(a)) | ((uint32_t)__bfloat16_as_ushort(bf(b)) << 16);
}

// One warp per voxel row: A row of the GEMM and ||yh||^2.
// ------------------------------------------------------------------ voxel order
// Voxels whose TACs are alike share their nearest draws, so the rare keys that
// pass the epilogue's threshold fall into the same columns for all of them.
// The fused kernel therefore processes voxels in an order that keeps such
// voxels in the same warp: a Morton key over three features (log of the
// weighted early, middle and late thirds of the TAC), counting-sorted on its
// top 16 bits.  Only the processing order changes; every voxel's result is
// computed exactly as before.
__device__ __forceinline__ uint32_t ord_f2u(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord_u2f(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// mm = {min, max} x 3 features as ordered integers; hist = 0
__global__ void k_order_init(uint32_t* __restrict__ mm, uint32_t* __restrict__ hist) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 6) mm[i] = (i & 1) ? 0u : 0xFFFFFFFFu;
    if (i < ORDER_BUCKETS) hist[i] = 0u;
}

// feat[3 j + c] = log of the weighted sum of third c of voxel j's TAC
__global__ void k_order_features(const float* __restrict__ y, int64_t J, int ldy, int L, Weights W,
                                 float* __restrict__ feat, uint32_t* __restrict__ mm) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    const float* yr = y + j * ldy;
    float f[3] = {0.0f, 0.0f, 0.0f};
    for (int l = 0; l < L; ++l) {
        const int c = (3 * l) / L;
        f[c] = fmaf(W.w[l], yr[l], f[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float v = logf(fmaxf(f[c], 1e-30f));
        feat[3 * j + c] = v;
        atomicMin(&mm[2 * c], ord_f2u(v));
        atomicMax(&mm[2 * c + 1], ord_f2u(v));
    }
}

__device__ __forceinline__ uint32_t spread3(uint32_t x) {     // bit i -> bit 3i (10 bits)
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__device__ __forceinline__ uint32_t order_key(const float* feat, const uint32_t* mm, int64_t j) {
    uint32_t q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float lo = ord_u2f(mm[2 * c]), hi = ord_u2f(mm[2 * c + 1]);
        const float t = hi > lo ? (feat[3 * j + c] - lo) / (hi - lo) : 0.0f;
        q[c] = (uint32_t)fminf(fmaxf(t * (float)((1 << ORDER_BITS) - 1), 0.0f), (float)((1 << ORDER_BITS) - 1));
    }
    return spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
}

// Counting-sort bucket of row j.  Draws (nlev > 0) are grouped first by the
// pilot samples they belong to: the draws j with j % s1^nlev == 0 (the coarsest
// pilot) come first, then those of the next finer pilot, and so on, so every
// pilot pass reads a contiguous leading block of the packed draws; within a
// group (but the coarsest) the Morton key orders them.  Voxels (nlev = 0):
// Morton key only.
__device__ __forceinline__ uint32_t order_bucket(const float* feat, const uint32_t* mm, int64_t j, int nlev,
                                                 int64_t s1) {
    const uint32_t key = order_key(feat, mm, j);
    if (nlev <= 0) return key >> (3 * ORDER_BITS - ORDER_BUCKET_BITS);
    int g = 0;
    int64_t sl = s1;
    for (int l = 1; l <= nlev; ++l, sl *= s1) g += (j % sl) == 0;
    // the coarsest pilot starts without a threshold and converges fastest on
    // draws in arbitrary order: its group is one bucket
    if (g == nlev) return 0u;
    return ((uint32_t)(nlev - g) << (ORDER_BUCKET_BITS - 3)) | (key >> (3 * ORDER_BITS - (ORDER_BUCKET_BITS - 3)));
}

__global__ void k_order_hist(const float* __restrict__ feat, const uint32_t* __restrict__ mm, int64_t J, int nlev,
                             int64_t s1, uint32_t* __restrict__ hist) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < J) atomicAdd(&hist[order_bucket(feat, mm, j, nlev, s1)], 1u);
}

// exclusive scan of the ORDER_BUCKETS counts, in place (one block of 1024 threads)
// Exclusive scan of the ORDER_BUCKETS bucket counts in three launches of
// coalesced 1024-entry blocks: block totals, a scan of the totals, then each
// block's scan plus its offset.
constexpr int SCAN_BLOCKS = ORDER_BUCKETS / 1024;

__device__ __forceinline__ uint32_t block_exclusive_scan_1024(uint32_t v, uint32_t* wsum, uint32_t& total) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[wp] = incl;
    __syncthreads();
    if (wp == 0) {
        const uint32_t x = wsum[lane];
        uint32_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, xi, o);
            if (lane >= o) xi += u;
        }
        wsum[lane] = xi - x;
        if (lane == 31) wsum[32] = xi;
    }
    __syncthreads();
    total = wsum[32];
    return wsum[wp] + incl - v;
}

__global__ void __launch_bounds__(1024) k_order_scan_sums(const uint32_t* __restrict__ hist, uint32_t* __restrict__ sums) {
    __shared__ uint32_t wsum[33];
    uint32_t total;
    block_exclusive_scan_1024(hist[blockIdx.x * 1024 + threadIdx.x], wsum, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_order_scan_top(uint32_t* __restrict__ sums) {
    __shared__ uint32_t wsum[33];
    uint32_t total;
    const uint32_t v = threadIdx.x < SCAN_BLOCKS ? sums[threadIdx.x] : 0u;
    const uint32_t e = block_exclusive_scan_1024(v, wsum, total);
    if (threadIdx.x < SCAN_BLOCKS) sums[threadIdx.x] = e;
}

__global__ void __launch_bounds__(1024) k_order_scan(uint32_t* __restrict__ hist, const uint32_t* __restrict__ sums) {
    __shared__ uint32_t wsum[33];
    uint32_t total;
    const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    const uint32_t e = block_exclusive_scan_1024(hist[i], wsum, total);
    hist[i] = sums[blockIdx.x] + e;
}

// perm[position] = voxel; voxels of one bucket land in arrival order
__global__ void k_order_scatter(const float* __restrict__ feat, const uint32_t* __restrict__ mm, int64_t J,
                                int nlev, int64_t s1, uint32_t* __restrict__ hist, int32_t* __restrict__ perm) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    const uint32_t pos = atomicAdd(&hist[order_bucket(feat, mm, j, nlev, s1)], 1u);
    perm[pos] = (int32_t)j;
}

// ABC_SPLIT_DRAWS also records, per voxel, the rounding of its bf16 row,
// delta = bf16(yh) - yh: c0 = -2 delta . yh and dn = ||delta|| (certificate).
// Weighted sums of the three consecutive thirds of a TAC (the features of the
// tile bound), computed by a warp; every lane gets them.
// ------------------------------------------------------------------ k-d order
// For a large scan the rows (the voxels; the draws of each pilot group) are ordered by a k-d
// split of their bound coordinates u_c = F_c / sqrt(W_c) (F_c the weighted sum over third c of
// the frames: the coordinates in which the tile bound measures gaps).  A run [a, b) of the
// order that contains a 128-row tile boundary splits its widest coordinate at the boundary
// nearest its middle, so every tile is one leaf, and its rows are those a median split put
// together: tighter tile boxes than runs of a space-filling curve.  The split value comes from
// a KD_BINS-bin histogram of the run's values on that coordinate; the rows of the bin holding
// the boundary go to either side by ticket.  Levels run breadth first; node n of level l has
// the children 2n and 2n + 1 (dense numbering; the roots are the pilot groups).
constexpr int KD_BINS = 128;
constexpr int KD_TILE = 128;
constexpr int KD_MAX_GROUPS = MAX_PILOT_LEVELS + 1;
constexpr double KD_MIN_PAIRS = 68719476736.0;   // 2^36 voxel-draw pairs: scans at least this large

struct KdNode {
    int32_t a, b;          // the run [a, b) of the order
    int32_t m;             // split position (a multiple of KD_TILE), b for a leaf
    int32_t dim;           // the widest coordinate
    float lo, inv;         // bin of a value v: (v - lo) inv, clamped to [0, KD_BINS)
    int32_t bstar, need;   // the bin holding the boundary, its rows that go left
    int32_t lcur, rcur, tick;
    uint32_t box[6];       // ordered-integer min, max per coordinate
};

struct KdGroups {
    int32_t start[KD_MAX_GROUPS + 1];   // group q holds positions [start[q], start[q + 1])
    int n;                              // groups
    int frozen;                         // a group kept in arbitrary order (the coarsest pilot's), or -1
    int nlev;                           // pilot levels (group q = nlev - pilot levels the row is in)
    int64_t s1;                         // pilot stride
    float isw[3];                       // 1 / sqrt(W_c)
};

__device__ __forceinline__ int kd_bin(float v, float lo, float inv) {
    const float t = (v - lo) * inv;
    return t >= 1.0f ? (int)fminf(t, (float)(KD_BINS - 1)) : 0;   // NaN and t < 1: bin 0
}

// an internal inconsistency (never expected): the outputs are flagged as not valid
__device__ __forceinline__ void kd_fail(int32_t* status) { atomicCAS(status, 0, ABC_ERR_UNSUPPORTED); }

// Bound coordinates of each row, its pilot group, and its place in the group's run (by ticket).
__global__ void k_kd_seed(const float* __restrict__ x, int64_t N, int ldx, int L, Weights W, KdGroups G,
                          int32_t* __restrict__ gcur, float4* __restrict__ kf, int32_t* __restrict__ krow,
                          int32_t* __restrict__ knode, int32_t* __restrict__ status) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = j < N;
    float F[3] = {0.0f, 0.0f, 0.0f};
    int q = -1;
    if (valid) {
        const float* r = x + j * ldx;
        for (int l = 0; l < L; ++l) {
            const int c = (3 * l) / L;
            const float v = W.w[l] * r[l];
            F[0] += c == 0 ? v : 0.0f;
            F[1] += c == 1 ? v : 0.0f;
            F[2] += c == 2 ? v : 0.0f;
        }
        int g = 0;
        int64_t sl = G.s1;
        for (int l = 1; l <= G.nlev; ++l, sl *= G.s1) g += (j % sl) == 0;
        q = G.nlev - g;
    }
    // tickets per group, one atomic per group present in the warp
    const uint32_t same = __match_any_sync(0xFFFFFFFFu, q);
    const int leader = __ffs(same) - 1;
    int base = 0;
    if (valid && lane == leader) base = atomicAdd(&gcur[q], __popc(same));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (!valid) return;
    const int64_t pos = (int64_t)G.start[q] + base + __popc(same & ((1u << lane) - 1u));
    if (pos >= G.start[q + 1]) {
        kd_fail(status);
        return;
    }
    kf[pos] = make_float4(F[0] * G.isw[0], F[1] * G.isw[1], F[2] * G.isw[2], 0.0f);
    krow[pos] = (int32_t)j;
    knode[pos] = q;
}

// Level roots: group q is node q of level 0.
__global__ void k_kd_roots(KdGroups G, KdNode* __restrict__ nd) {
    const int q = threadIdx.x;
    if (q < G.n) {
        nd[q].a = G.start[q];
        nd[q].b = G.start[q + 1];
    }
}

// Clears the boxes, cursors and histograms of the nn nodes of a level.
__global__ void k_kd_level_init(KdNode* __restrict__ nd, uint32_t* __restrict__ hist, int64_t nn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nn * KD_BINS) hist[i] = 0u;
    if (i < nn) {
        KdNode& n = nd[i];
        for (int c = 0; c < 3; ++c) {
            n.box[2 * c] = 0xFFFFFFFFu;
            n.box[2 * c + 1] = 0u;
        }
        n.lcur = n.rcur = n.tick = 0;
        n.m = n.b;
    }
}

// Node boxes.  The runs are contiguous and sorted by node, so a block whose first and last
// rows share a node holds that node alone: it reduces its rows in shared memory and issues one
// set of atomics (the top levels, where every block of the level hits the same few nodes);
// otherwise one set per warp whose rows share a node, else one per row.
__global__ void __launch_bounds__(256) k_kd_box(const float4* __restrict__ kf, const int32_t* __restrict__ knode,
                                                int64_t N, KdNode* __restrict__ nd) {
    __shared__ uint32_t sred[8][6];
    const int64_t p0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t p = p0 + threadIdx.x;
    const int64_t plast = (p0 + blockDim.x <= N ? p0 + blockDim.x : N) - 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool valid = p < N;
    const int node = valid ? knode[p] : -1;
    float f[3] = {0.0f, 0.0f, 0.0f};
    if (valid) {
        const float4 v = kf[p];
        f[0] = v.x;
        f[1] = v.y;
        f[2] = v.z;
    }
    const int nb = knode[p0];
    if (nb == knode[plast]) {
        // rows past N take the identities of min and max
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint32_t u = ord_f2u(f[c]);
            const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, valid ? u : 0xFFFFFFFFu);
            const uint32_t mx = __reduce_max_sync(0xFFFFFFFFu, valid ? u : 0u);
            if (lane == 0) {
                sred[wid][2 * c] = mn;
                sred[wid][2 * c + 1] = mx;
            }
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            const int e = threadIdx.x;
            const int nw = blockDim.x >> 5;
            uint32_t v = sred[0][e];
            for (int w = 1; w < nw; ++w) v = (e & 1) ? max(v, sred[w][e]) : min(v, sred[w][e]);
            if (e & 1) atomicMax(&nd[nb].box[e], v);
            else atomicMin(&nd[nb].box[e], v);
        }
        return;
    }
    const int n0 = __shfl_sync(0xFFFFFFFFu, node, 0);
    if (__all_sync(0xFFFFFFFFu, valid && node == n0)) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint32_t u = ord_f2u(f[c]);
            const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, u), mx = __reduce_max_sync(0xFFFFFFFFu, u);
            if (lane == 0) {
                atomicMin(&nd[n0].box[2 * c], mn);
                atomicMax(&nd[n0].box[2 * c + 1], mx);
            }
        }
    } else if (valid) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicMin(&nd[node].box[2 * c], ord_f2u(f[c]));
            atomicMax(&nd[node].box[2 * c + 1], ord_f2u(f[c]));
        }
    }
}

// Per node of level `level`: whether it splits (it holds a tile boundary and is not in the
// frozen group), where, and along which coordinate.
__global__ void k_kd_dims(KdNode* __restrict__ nd, int64_t nn, int level, int frozen) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    KdNode& n = nd[i];
    const int32_t a = n.a, b = n.b;
    const int32_t first = (a / KD_TILE + 1) * KD_TILE;   // the first boundary past a
    if (first >= b || (frozen >= 0 && (i >> level) == frozen)) {
        n.m = b;
        return;
    }
    int d = 0;
    float best = -1.0f, lo = 0.0f;
    for (int c = 0; c < 3; ++c) {
        const float l = ord_u2f(n.box[2 * c]), h = ord_u2f(n.box[2 * c + 1]);
        const float w = h - l;
        if (w > best) {
            best = w;
            d = c;
            lo = l;
        }
    }
    n.dim = d;
    n.lo = lo;
    n.inv = (best > 0.0f && best < 3.0e38f) ? (float)KD_BINS / best : 0.0f;
    const int32_t last = ((b - 1) / KD_TILE) * KD_TILE;   // the last boundary before b
    int32_t m = (int32_t)((((int64_t)a + b) / 2 + KD_TILE / 2) / KD_TILE) * KD_TILE;
    n.m = m < first ? first : (m > last ? last : m);
}

// Histogram of each splitting node's values on its coordinate: in shared memory for a block
// whose rows share one node (the runs are contiguous), else in global memory.
__global__ void __launch_bounds__(256) k_kd_hist(const float4* __restrict__ kf, const int32_t* __restrict__ knode,
                                                 int64_t N, const KdNode* __restrict__ nd,
                                                 uint32_t* __restrict__ hist) {
    __shared__ uint32_t sh[KD_BINS];
    const int64_t p0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t p = p0 + threadIdx.x;
    const int64_t plast = (p0 + blockDim.x <= N ? p0 + blockDim.x : N) - 1;
    const bool uni = knode[p0] == knode[plast];
    if (uni)
        for (int i = threadIdx.x; i < KD_BINS; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    if (p < N) {
        const int node = knode[p];
        const KdNode& n = nd[node];
        if (n.m < n.b) {
            const float4 v = kf[p];
            const float u = n.dim == 0 ? v.x : (n.dim == 1 ? v.y : v.z);
            const int bin = kd_bin(u, n.lo, n.inv);
            if (uni) atomicAdd(&sh[bin], 1u);
            else atomicAdd(&hist[(int64_t)node * KD_BINS + bin], 1u);
        }
    }
    __syncthreads();
    if (uni) {
        const int node = knode[p0];
        for (int i = threadIdx.x; i < KD_BINS; i += blockDim.x)
            if (sh[i]) atomicAdd(&hist[(int64_t)node * KD_BINS + i], sh[i]);
    }
}

// One warp per node: the bin holding the split position and the count of its rows that go
// left; the children's runs for the next level (a leaf passes its run to child 2n).
__global__ void k_kd_split(KdNode* __restrict__ nd, const uint32_t* __restrict__ hist, int64_t nn,
                           KdNode* __restrict__ nx, int32_t* __restrict__ status) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= nn) return;
    KdNode& n = nd[i];
    const int32_t a = n.a, b = n.b, m = n.m;
    if (lane == 0) {
        nx[2 * i].a = a;
        nx[2 * i].b = m;
        nx[2 * i + 1].a = m;
        nx[2 * i + 1].b = b;
    }
    if (m >= b) return;
    const int target = m - a;
    uint32_t h[KD_BINS / 32], sum = 0;
#pragma unroll
    for (int q = 0; q < KD_BINS / 32; ++q) {
        h[q] = hist[i * KD_BINS + lane * (KD_BINS / 32) + q];
        sum += h[q];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t c = incl - sum;
    int found = -1, below = 0;
#pragma unroll
    for (int q = 0; q < KD_BINS / 32; ++q) {
        if (found < 0 && c + h[q] >= (uint32_t)target) {
            found = lane * (KD_BINS / 32) + q;
            below = (int)c;
        }
        c += h[q];
    }
    const uint32_t who = __ballot_sync(0xFFFFFFFFu, found >= 0);
    if (total != (uint32_t)(b - a) || !who) {
        if (lane == 0) kd_fail(status);
        return;
    }
    const int src = __ffs(who) - 1;
    if (lane == src) {
        n.bstar = found;
        n.need = target - below;
    }
}

// Rows to their child runs: below the boundary's bin left, above it right, and in it by
// ticket (the first `need` tickets left).  A block whose rows share one splitting node (the
// runs are contiguous) reserves its tickets and places with one atomic per counter; otherwise
// one set per warp whose rows share a node, else per row.  A leaf's rows keep their places.
__global__ void __launch_bounds__(256) k_kd_scatter(const float4* __restrict__ kf, const int32_t* __restrict__ krow,
                                                    const int32_t* __restrict__ knode, int64_t N,
                                                    KdNode* __restrict__ nd, float4* __restrict__ kf2,
                                                    int32_t* __restrict__ krow2, int32_t* __restrict__ knode2,
                                                    int32_t* __restrict__ status) {
    __shared__ int s_cnt[3][8];    // per warp: rows in the boundary's bin, rows going left, right
    __shared__ int s_base[3][8];   // their first ticket / place
    const int64_t p0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t p = p0 + threadIdx.x;
    const int64_t plast = (p0 + blockDim.x <= N ? p0 + blockDim.x : N) - 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const bool valid = p < N;
    const int node = valid ? knode[p] : -1;
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int32_t a = 0, b = 0, m = 0;
    int cls = -1;   // -1: stays (leaf), 0: left, 1: right, 2: the boundary's bin
    if (valid) {
        v = kf[p];
        const KdNode& n = nd[node];
        a = n.a;
        b = n.b;
        m = n.m;
        if (m < b) {
            const float u = n.dim == 0 ? v.x : (n.dim == 1 ? v.y : v.z);
            const int bin = kd_bin(u, n.lo, n.inv);
            cls = bin < n.bstar ? 0 : (bin > n.bstar ? 1 : 2);
        }
    }
    int64_t pos = p;
    const int nb = knode[p0];
    if (nb == knode[plast]) {
        // every row of the block is in node nb; a leaf's rows stay
        KdNode& n = nd[nb];
        if (n.m < n.b) {
            const int nw = blockDim.x >> 5;
            const uint32_t tm = __ballot_sync(0xFFFFFFFFu, valid && cls == 2);
            if (lane == 0) s_cnt[0][wid] = __popc(tm);
            __syncthreads();
            if (threadIdx.x == 0) {
                int tot = 0;
                for (int w = 0; w < nw; ++w) {
                    s_base[0][w] = tot;
                    tot += s_cnt[0][w];
                }
                const int tb = tot ? atomicAdd(&n.tick, tot) : 0;
                for (int w = 0; w < nw; ++w) s_base[0][w] += tb;
            }
            __syncthreads();
            if (cls == 2) cls = (s_base[0][wid] + __popc(tm & lt)) < n.need ? 0 : 1;
            const uint32_t lm = __ballot_sync(0xFFFFFFFFu, valid && cls == 0);
            const uint32_t rm = __ballot_sync(0xFFFFFFFFu, valid && cls == 1);
            if (lane == 0) {
                s_cnt[1][wid] = __popc(lm);
                s_cnt[2][wid] = __popc(rm);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int tl = 0, tr = 0;
                for (int w = 0; w < nw; ++w) {
                    s_base[1][w] = tl;
                    tl += s_cnt[1][w];
                    s_base[2][w] = tr;
                    tr += s_cnt[2][w];
                }
                const int lb = tl ? atomicAdd(&n.lcur, tl) : 0;
                const int rb = tr ? atomicAdd(&n.rcur, tr) : 0;
                for (int w = 0; w < nw; ++w) {
                    s_base[1][w] += lb;
                    s_base[2][w] += rb;
                }
            }
            __syncthreads();
            if (valid)
                pos = cls == 0 ? (int64_t)a + s_base[1][wid] + __popc(lm & lt)
                               : (int64_t)m + s_base[2][wid] + __popc(rm & lt);
        }
    } else {
        const int n0 = __shfl_sync(0xFFFFFFFFu, node, 0);
        const bool uni = __all_sync(0xFFFFFFFFu, valid && node == n0);
        if (uni && cls >= 0) {   // the whole warp: one node that splits
            KdNode& n = nd[n0];
            const uint32_t tm = __ballot_sync(0xFFFFFFFFu, cls == 2);
            int tb = 0;
            if (lane == 0 && tm) tb = atomicAdd(&n.tick, __popc(tm));
            tb = __shfl_sync(0xFFFFFFFFu, tb, 0);
            if (cls == 2) cls = (tb + __popc(tm & lt)) < n.need ? 0 : 1;
            const uint32_t lm = __ballot_sync(0xFFFFFFFFu, cls == 0), rm = ~lm;
            int lb = 0, rb = 0;
            if (lane == 0) {
                if (lm) lb = atomicAdd(&n.lcur, __popc(lm));
                if (rm) rb = atomicAdd(&n.rcur, __popc(rm));
            }
            lb = __shfl_sync(0xFFFFFFFFu, lb, 0);
            rb = __shfl_sync(0xFFFFFFFFu, rb, 0);
            pos = cls == 0 ? (int64_t)a + lb + __popc(lm & lt) : (int64_t)m + rb + __popc(rm & lt);
        } else if (valid && cls >= 0) {
            KdNode& n = nd[node];
            if (cls == 2) cls = atomicAdd(&n.tick, 1) < n.need ? 0 : 1;
            pos = cls == 0 ? (int64_t)a + atomicAdd(&n.lcur, 1) : (int64_t)m + atomicAdd(&n.rcur, 1);
        }
    }
    if (!valid) return;
    const int side = cls == 1 ? 1 : 0;
    if (pos < (side ? m : a) || pos >= (cls < 0 ? b : (side ? b : m))) {
        kd_fail(status);
        return;
    }
    kf2[pos] = v;
    krow2[pos] = krow[p];
    knode2[pos] = 2 * node + side;
}

__global__ void k_kd_copy(const int32_t* __restrict__ src, int64_t N, int32_t* __restrict__ dst) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) dst[p] = src[p];
}

// Orders the N rows of x (row stride ldx) by the k-d split into perm (perm[p] = the row at
// position p); with nlev > 0 the rows are first grouped by pilot level like the Morton
// order (the coarsest pilot's group first and left in arbitrary order).  The work arrays
// live in `scratch` (a buffer written only later in the call); done = false, nothing
// launched, when it does not hold them.
int kd_order(const float* x, int64_t N, int ldx, int L, const Weights& W, int nlev, int64_t s1, void* scratch,
             size_t scratch_bytes, int32_t* perm, int32_t* status, cudaStream_t s, bool& done) {
    done = false;
    if (N < 2 * KD_TILE || N >= ((int64_t)1 << 30) || nlev + 1 > KD_MAX_GROUPS) return ABC_OK;
    KdGroups G;
    memset(&G, 0, sizeof G);
    G.nlev = nlev;
    G.s1 = s1 > 1 ? s1 : 2;
    G.n = nlev + 1;
    G.frozen = nlev > 0 ? 0 : -1;
    // group q holds the rows in nlev - q pilot samples: ceil(N / s1^l) rows are in sample l
    int64_t in_sample[KD_MAX_GROUPS + 1];
    int64_t sl = 1;
    for (int l = 0; l <= nlev; ++l, sl *= G.s1) in_sample[l] = (N + sl - 1) / sl;
    in_sample[nlev + 1] = 0;
    G.start[0] = 0;
    for (int q = 0; q < G.n; ++q) {
        const int g = nlev - q;   // pilot samples of the group's rows
        const int64_t size = in_sample[g] - (g < nlev ? in_sample[g + 1] : 0);
        G.start[q + 1] = (int32_t)(G.start[q] + size);
    }
    for (int c = 0; c < 3; ++c) {
        double wc = 0.0;
        for (int l = 0; l < L; ++l)
            if ((3 * l) / L == c) wc += W.w[l];
        G.isw[c] = wc > 0.0 ? (float)(1.0 / sqrt(wc)) : 0.0f;
    }
    // levels: every run of a group that holds a tile boundary halves its tiles per level
    int levels = 0;
    for (int q = 0; q < G.n; ++q) {
        if (q == G.frozen || G.start[q + 1] <= G.start[q]) continue;
        const int64_t pieces = (G.start[q + 1] - 1) / KD_TILE - G.start[q] / KD_TILE + 1;
        int lv = 0;
        while (((int64_t)1 << lv) < pieces) ++lv;
        levels = lv > levels ? lv : levels;
    }
    if (levels == 0) return ABC_OK;
    const int64_t nn_max = (int64_t)G.n << levels;   // nodes of the deepest table
    // scratch: rows (two copies), node tables (two), histograms (a splitting level's)
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = (o + bytes + 255) & ~(size_t)255; return at; };
    const size_t o_kf0 = take((size_t)N * 16), o_kf1 = take((size_t)N * 16);
    const size_t o_r0 = take((size_t)N * 4), o_r1 = take((size_t)N * 4);
    const size_t o_n0 = take((size_t)N * 4), o_n1 = take((size_t)N * 4);
    const size_t o_g = take(KD_MAX_GROUPS * 4);
    const size_t o_d0 = take((size_t)nn_max * sizeof(KdNode)), o_d1 = take((size_t)nn_max * sizeof(KdNode));
    const size_t o_h = take((size_t)(nn_max / 2) * KD_BINS * 4);
    if (o > scratch_bytes) return ABC_OK;
    uint8_t* sb = (uint8_t*)scratch;
    float4* kf[2] = {(float4*)(sb + o_kf0), (float4*)(sb + o_kf1)};
    int32_t* kr[2] = {(int32_t*)(sb + o_r0), (int32_t*)(sb + o_r1)};
    int32_t* kn[2] = {(int32_t*)(sb + o_n0), (int32_t*)(sb + o_n1)};
    int32_t* gcur = (int32_t*)(sb + o_g);
    KdNode* nd[2] = {(KdNode*)(sb + o_d0), (KdNode*)(sb + o_d1)};
    uint32_t* hist = (uint32_t*)(sb + o_h);
    const unsigned gb = (unsigned)vpet_ceil_div(N, 256);
    VPET_CUDA(cudaMemsetAsync(gcur, 0, KD_MAX_GROUPS * 4, s));
    k_kd_seed<<<gb, 256, 0, s>>>(x, N, ldx, L, W, G, gcur, kf[0], kr[0], kn[0], status);
    VPET_LAUNCH_CHECK();
    k_kd_roots<<<1, 32, 0, s>>>(G, nd[0]);
    VPET_LAUNCH_CHECK();
    int c = 0;
    for (int l = 0; l < levels; ++l) {
        const int64_t nn = (int64_t)G.n << l;
        k_kd_level_init<<<(unsigned)vpet_ceil_div(nn * KD_BINS, 256), 256, 0, s>>>(nd[c], hist, nn);
        VPET_LAUNCH_CHECK();
        k_kd_box<<<gb, 256, 0, s>>>(kf[c], kn[c], N, nd[c]);
        VPET_LAUNCH_CHECK();
        k_kd_dims<<<(unsigned)vpet_ceil_div(nn, 256), 256, 0, s>>>(nd[c], nn, l, G.frozen);
        VPET_LAUNCH_CHECK();
        k_kd_hist<<<gb, 256, 0, s>>>(kf[c], kn[c], N, nd[c], hist);
        VPET_LAUNCH_CHECK();
        k_kd_split<<<(unsigned)vpet_ceil_div(nn * 32, 256), 256, 0, s>>>(nd[c], hist, nn, nd[1 - c], status);
        VPET_LAUNCH_CHECK();
        k_kd_scatter<<<gb, 256, 0, s>>>(kf[c], kr[c], kn[c], N, nd[c], kf[1 - c], kr[1 - c], kn[1 - c], status);
        VPET_LAUNCH_CHECK();
        c = 1 - c;
    }
    k_kd_copy<<<gb, 256, 0, s>>>(kr[c], N, perm);
    VPET_LAUNCH_CHECK();
    done = true;
    return ABC_OK;
}

__device__ __forceinline__ void seg_features(const float* r, int L, const float* w, int lane, float (&f)[3]) {
    f[0] = f[1] = f[2] = 0.0f;
    for (int l = lane; l < L; l += 32) {
        const int c = (3 * l) / L;
        const float v = w[l] * r[l];
        f[0] += c == 0 ? v : 0.0f;
        f[1] += c == 1 ? v : 0.0f;
        f[2] += c == 2 ? v : 0.0f;
    }
    f[0] = warp_sum(f[0]);
    f[1] = warp_sum(f[1]);
    f[2] = warp_sum(f[2]);
}

// The frame weights, their square roots and the centring means in shared memory:
// read by lane-varying frame index, which the kernel parameter space would
// serialise across the warp.
struct FrameConsts {
    float w[MAXL], sw[MAXL], mu[MAXL];
};

__device__ __forceinline__ void stage_frame_consts(FrameConsts& S, const Weights& W, const float* mu, int L) {
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        S.w[l] = W.w[l];
        S.sw[l] = W.sw[l];
        S.mu[l] = mu[l];
    }
    __syncthreads();
}

// Row j of A is voxel perm[j] (perm = null: voxel j); fy[3 j + c] = its segment features.
// mu: the groups' means (MAXL each); a block's 8 rows lie in one group (Jg is a multiple of 128).
__global__ void k_pack_y(const float* __restrict__ y, int64_t J, int64_t Jp, int ldy, int L, int Kp, int mode,
                         Weights W, const float* __restrict__ mu, int64_t Jg, const int32_t* __restrict__ perm,
                         __nv_bfloat16* __restrict__ A, float* __restrict__ ynorm, float* __restrict__ c0,
                         float* __restrict__ dn, float* __restrict__ fy) {
    __shared__ FrameConsts F;
    stage_frame_consts(F, W, mu + ((int64_t)blockIdx.x * (blockDim.x >> 5) / Jg) * MAXL, L);
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= Jp) return;
    __nv_bfloat16* row = A + j * Kp;
    if (j >= J) {
        for (int e = lane; e < Kp; e += 32) row[e] = bf(0.0f);
        if (lane == 0) {
            ynorm[j] = 0.0f;
            c0[j] = 0.0f;
            dn[j] = 0.0f;
        }
        return;
    }
    const float* yr = y + (perm ? (int64_t)perm[j] : j) * ldy;
    float ss = 0.0f, sc = 0.0f, sd = 0.0f;
    for (int l = lane; l < L; l += 32) {
        const float v = F.sw[l] * (yr[l] - F.mu[l]);
        ss = fmaf(v, v, ss);
        const float dl = __bfloat162float(bf(v)) - v;       // exact in fp32
        sc = fmaf(dl, v, sc);
        sd = fmaf(dl, dl, sd);
    }
    ss = warp_sum(ss);
    sc = warp_sum(sc);
    sd = warp_sum(sd);
    float f[3];
    seg_features(yr, L, F.w, lane, f);
    if (lane == 0) {
        ynorm[j] = ss;
        c0[j] = -2.0f * sc;
        dn[j] = sqrtf(sd);
        fy[3 * j] = f[0];
        fy[3 * j + 1] = f[1];
        fy[3 * j + 2] = f[2];
    }
    for (int e = lane; e < Kp; e += 32) {
        float out = 0.0f;
        if (mode == ABC_FP32) {
            if (e < 3 * L) {
                const int l = e % L;
                const float v = F.sw[l] * (yr[l] - F.mu[l]);
                const float hi = __bfloat162float(bf(v));
                out = e < 2 * L ? hi : v - hi;
            } else if (e < 3 * L + 3) {
                out = 1.0f;
            }
        } else {
            if (e < 2 * L) {
                const int l = e % L;
                out = F.sw[l] * (yr[l] - F.mu[l]);              // the same bf16 row against x_hi and x_lo
            } else if (e < 2 * L + 3) {
                out = 1.0f;
            }
        }
        row[e] = bf(out);
    }
}

// One warp per four draw rows: B rows of the GEMM.
// Row n of B is draw xperm[n] (xperm = null: draw n); fx[3 n + c] = its segment
// features; xs row n (stride ldxs, zero-padded) = that draw's fp32 TAC, so that
// the exact re-score reads the draws in packed order.  The warp's four source
// rows are read into shared memory with all their loads in flight together.
constexpr int PACK_ROWS = 4;
constexpr int PACK_KMAX = 256;                 // widest packed row (3 x 64 frames + 3 norm columns)
constexpr int MAX_GROUPS = 16;                 // centring groups per scan
// B holds G copies of the packed draws, copy g (rows [g Np, (g+1) Np)) centred on group
// g's mean mu[g]; the fp32 copy xs and the segment features are written once.
__global__ void __launch_bounds__(256) k_pack_x(const float* __restrict__ x, int64_t N, int64_t Np, int ldx, int L,
                                                int Kp, int mode, Weights W, const float* __restrict__ mu, int G,
                                                const int32_t* __restrict__ xperm, __nv_bfloat16* __restrict__ B,
                                                float* __restrict__ fx, float* __restrict__ xs, int ldxs) {
    __shared__ FrameConsts F;
    __shared__ __align__(16) float s_mu[MAX_GROUPS][MAXL];
    __shared__ float s_rows[8][PACK_ROWS][MAXL];
    __shared__ __align__(16) __nv_bfloat16 s_rowbuf[8][PACK_KMAX];
    for (int e = threadIdx.x; e < G * MAXL; e += blockDim.x) s_mu[e / MAXL][e % MAXL] = mu[e];
    stage_frame_consts(F, W, mu, L);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // Each lane owns the frame pair l0 = 2 lane, l1 = l0 + 1 (zero weight past L); a
    // packed row is assembled in the warp's row buffer (bf16, Kp columns; its columns past
    // the norm parts stay zero) and leaves as 16-byte stores.
    const int l0 = 2 * lane, l1 = l0 + 1;
    const float sw0 = l0 < L ? F.sw[l0] : 0.0f, sw1 = l1 < L ? F.sw[l1] : 0.0f;
    __nv_bfloat16* rb = s_rowbuf[wid];
    const int aug = cols_per_frame(mode) * L;
    for (int e = lane; e < Kp; e += 32) rb[e] = bf(0.0f);
    __syncwarp();
    const int64_t nb = ((int64_t)blockIdx.x * 8 + wid) * PACK_ROWS;
    if (nb >= Np) return;
    {
        int64_t src[PACK_ROWS];
#pragma unroll
        for (int u = 0; u < PACK_ROWS; ++u) {
            const int64_t n = nb + u;
            src[u] = n < N ? (xperm ? (int64_t)xperm[n] : n) : -1;
        }
        float v[PACK_ROWS][2];
#pragma unroll
        for (int u = 0; u < PACK_ROWS; ++u)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int l = lane + 32 * q;
                v[u][q] = (src[u] >= 0 && l < L) ? x[src[u] * ldx + l] : 0.0f;
            }
#pragma unroll
        for (int u = 0; u < PACK_ROWS; ++u)
#pragma unroll
            for (int q = 0; q < 2; ++q) s_rows[wid][u][lane + 32 * q] = v[u][q];
        __syncwarp();
    }
    for (int u = 0; u < PACK_ROWS; ++u) {
        const int64_t n = nb + u;
        if (n >= Np) break;
        if (n >= N) {
            for (int g = 0; g < G; ++g) {
                uint2* row = (uint2*)(B + ((int64_t)g * Np + n) * Kp);
                for (int e = lane; e < Kp / 4; e += 32) row[e] = make_uint2(0u, 0u);
            }
            continue;
        }
        const float* xr = s_rows[wid][u];
        for (int l = lane; l < ldxs; l += 32) xs[n * ldxs + l] = l < L ? xr[l] : 0.0f;
        {
            float f[3];
            seg_features(xr, L, F.w, lane, f);
            if (lane == 0) {
                fx[3 * n] = f[0];
                fx[3 * n + 1] = f[1];
                fx[3 * n + 2] = f[2];
            }
        }
        const float x0 = xr[l0], x1 = xr[l1];
        for (int g = 0; g < G; ++g) {
            const float2 m = *(const float2*)&s_mu[g][l0];
            const float v0 = sw0 * (x0 - m.x), v1 = sw1 * (x1 - m.y);
            const __nv_bfloat162 hp = __floats2bfloat162_rn(v0, v1);
            const float h0 = __low2float(hp), h1 = __high2float(hp);
            const float d0 = v0 - h0, d1 = v1 - h1;
            const __nv_bfloat162 lp = __floats2bfloat162_rn(d0, d1);
            float ss = fmaf(v1, v1, v0 * v0);
            // split form: b.r with r = v - hi - lo, exact in fp32
            float sr = fmaf(v1, d1 - __high2float(lp), v0 * (d0 - __low2float(lp)));
            // -2 hi and -2 lo are exact in bf16
            const __nv_bfloat162 ho = __floats2bfloat162_rn(-2.0f * h0, -2.0f * h1);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(-2.0f * __low2float(lp), -2.0f * __high2float(lp));
            if (l1 < L) {
                *(__nv_bfloat162*)&rb[l0] = ho;                       // 4-byte aligned (l0 even)
                rb[L + l0] = __low2bfloat16(lo);
                rb[L + l1] = __high2bfloat16(lo);
                if (mode == ABC_FP32) {
                    rb[2 * L + l0] = __low2bfloat16(ho);
                    rb[2 * L + l1] = __high2bfloat16(ho);
                }
            } else if (l0 < L) {
                rb[l0] = __low2bfloat16(ho);
                rb[L + l0] = __low2bfloat16(lo);
                if (mode == ABC_FP32) rb[2 * L + l0] = __low2bfloat16(ho);
            }
            ss = warp_sum(ss);
            // split form: the norm column carries ||b||^2 - 2 b.r, so that the key's error from the
            // draw row's split is 2 (a - b).r, which vanishes with the distance
            if (mode != ABC_FP32) ss -= 2.0f * warp_sum(sr);
            if (lane == 0) {
                const float n1 = __bfloat162float(bf(ss));
                const float r1 = ss - n1;
                const float n2 = __bfloat162float(bf(r1));
                rb[aug] = bf(n1);
                rb[aug + 1] = bf(n2);
                rb[aug + 2] = bf(r1 - n2);
            }
            __syncwarp();
            if (lane < Kp / 8)
                ((uint4*)(B + ((int64_t)g * Np + n) * Kp))[lane] = ((const uint4*)rb)[lane];
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------ tile bound
// For the weighted sums F_c(v) = sum_{l in third c} w_l v_l of the three thirds of
// the frames, Cauchy-Schwarz gives (F_c(y) - F_c(x))^2 <= W_c sum_{l in c} w_l (y_l - x_l)^2
// with W_c = sum_{l in c} w_l, so d(y, x) >= sum_c (F_c(y) - F_c(x))^2 / W_c.  With
// boxes [lo_c, hi_c] of the features over a 128-voxel tile and over a draw tile,
// the squared gaps between the boxes bound every pair of the two tiles from below.
// A draw tile whose bound exceeds the largest distance threshold of the voxel
// tile holds no draw that any of its voxels would keep, so the main pass skips it.

// tbox[6 t + 2 c], tbox[6 t + 2 c + 1] = min, max of feature c over the draws of 64-draw tile t
__global__ void k_tile_boxes(const float* __restrict__ fx, int64_t N, int64_t nt64, float* __restrict__ tbox) {
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= nt64) return;
    float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t n = t * 64 + h * 32 + lane;
        if (n < N) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                lo[c] = fminf(lo[c], fx[3 * n + c]);
                hi[c] = fmaxf(hi[c], fx[3 * n + c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xFFFFFFFFu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xFFFFFFFFu, hi[c], o));
        }
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            tbox[6 * t + 2 * c] = lo[c];
            tbox[6 * t + 2 * c + 1] = hi[c];
        }
}

struct KeepArgs {
    const float* fy;             // packed voxel rows x 3
    const float* thr0;           // key threshold per packed row (null: none, every tile is kept)
    const float* ynorm;          // ||yh||^2 per packed row
    const float* tbox;           // 64-draw tile boxes
    int32_t* ktile;              // kept tile indices, nvt x nt64 (row stride nt64)
    int32_t* kcount;             // kept tiles per voxel tile
    unsigned long long* tally;   // [0] += kept, [1] += all (diagnostics)
    int64_t J, N, nt64;
    float Wc[3];                 // segment weight sums
    float cE;                    // ABC_FP32: error coefficient of the keys
    int split;                   // split form: thresholds become distances by dist_ub
    SplitCoef sc;
    const float* c0;             // split form: per packed row
    const float* dn;
    const int32_t* rows;         // rescue pass: list row of each voxel position (thr0 is positional), or null
    const int32_t* count;        // rescue pass: queued voxels
    int bn;                      // draw-tile width of the pass, 64 or 128
    int order;                   // list a voxel tile's kept tiles nearest first (at most KEEP_SORT_MAX)
};

// Kept-tile lists up to this long can be put in nearest-first order (a pilot's).
constexpr int KEEP_SORT_MAX = 4096;

// One block (256 threads) per 128-voxel tile: the voxel tile's feature box and
// largest distance threshold, then the list of draw tiles that cannot be skipped,
// in draw order, or (order) by the distance between the centres of the voxel tile's
// box and the draw tile's: a pilot that meets the nearest draws first keeps its
// smallest keys early and rejects most later keys by its group-minimum test.
__global__ void __launch_bounds__(256) k_keep_tiles(const __grid_constant__ KeepArgs K) {
    __shared__ uint32_t box[7];                 // ordered-int min/max x 3, max threshold
    __shared__ int wcount[8];
    __shared__ unsigned long long sk[KEEP_SORT_MAX];   // (centre distance, tile) of the kept tiles
    // per voxel (packed order; td = -1: no voxel): its features widened by their rounding slack
    // (f - s, f + s) and its distance bound; per 16 consecutive voxels their box and largest bound
    __shared__ float4 sv_lo[BM], sv_hi[BM];
    __shared__ float4 sb_lo[BM / 16], sb_hi[BM / 16];
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const int64_t vt = blockIdx.x;
    const int64_t nv = K.count ? (int64_t)*K.count : K.J;   // voxel positions in use
    if (vt * BM >= nv) {
        if (tid == 0) K.kcount[vt] = 0;
        return;
    }
    if (tid < 7) box[tid] = (tid < 6 && (tid & 1) == 0) ? 0xFFFFFFFFu : 0u;
    __syncthreads();
    if (tid < BM) {
        sv_lo[tid] = make_float4(3.0e38f, 3.0e38f, 3.0e38f, -1.0f);
        sv_hi[tid] = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.0f);
        const int64_t p = vt * BM + tid;
        const int64_t j = K.rows && p < nv ? (int64_t)K.rows[p] : p;   // packed row of the voxel (-1: none)
        if (p < nv && p < K.J && j >= 0) {
            const float t = K.thr0 ? K.thr0[p] : 3.0e38f;
            const float yn = K.ynorm[j];
            float td;
            if (!K.thr0) {
                td = 3.0e38f;
            } else if (K.split) {
                // every draw whose key can pass t lies within this distance
                td = dist_ub(t, yn, K.c0[j], K.dn[j], K.sc);
            } else {
                td = t + yn;
                if (td < 1.0e30f) {
                    const float ry = sqrtf(fmaxf(yn, 0.0f));
                    const float R = ry + sqrtf(fmaxf(td, 0.0f));
                    td += K.cE * (2.0f * ry * R + R * R);
                }
            }
            td = td >= 1.0e30f ? 3.0e38f : td * (1.0f + 0x1p-10f) + 1e-30f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                atomicMin(&box[2 * c], ord_f2u(K.fy[3 * j + c]));
                atomicMax(&box[2 * c + 1], ord_f2u(K.fy[3 * j + c]));
            }
            atomicMax(&box[6], ord_f2u(td));
            float f[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) f[c] = K.fy[3 * j + c];
            // the voxel's share of the features' rounding slack, 2^-18 x 2 |f|
            sv_lo[tid] = make_float4(f[0] - 0x1p-17f * fabsf(f[0]), f[1] - 0x1p-17f * fabsf(f[1]),
                                     f[2] - 0x1p-17f * fabsf(f[2]), td);
            sv_hi[tid] = make_float4(f[0] + 0x1p-17f * fabsf(f[0]), f[1] + 0x1p-17f * fabsf(f[1]),
                                     f[2] + 0x1p-17f * fabsf(f[2]), 0.0f);
        }
        // the 16-voxel sub-boxes (half-warp reductions)
        float4 lo = sv_lo[tid], hi = sv_hi[tid];
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            lo.x = fminf(lo.x, __shfl_xor_sync(0xFFFFFFFFu, lo.x, o));
            lo.y = fminf(lo.y, __shfl_xor_sync(0xFFFFFFFFu, lo.y, o));
            lo.z = fminf(lo.z, __shfl_xor_sync(0xFFFFFFFFu, lo.z, o));
            lo.w = fmaxf(lo.w, __shfl_xor_sync(0xFFFFFFFFu, lo.w, o));
            hi.x = fmaxf(hi.x, __shfl_xor_sync(0xFFFFFFFFu, hi.x, o));
            hi.y = fmaxf(hi.y, __shfl_xor_sync(0xFFFFFFFFu, hi.y, o));
            hi.z = fmaxf(hi.z, __shfl_xor_sync(0xFFFFFFFFu, hi.z, o));
        }
        if ((tid & 15) == 0) {
            sb_lo[tid >> 4] = lo;
            sb_hi[tid >> 4] = hi;
        }
    }
    __syncthreads();
    float ylo[3], yhi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ylo[c] = ord_u2f(box[2 * c]);
        yhi[c] = ord_u2f(box[2 * c + 1]);
    }
    const float tmax = ord_u2f(box[6]);
    const bool all = !(tmax < 1.0e30f);
    float invW[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) invW[c] = K.Wc[c] > 0.0f ? 1.0f / K.Wc[c] : 0.0f;
    const int per = K.bn / 64;
    const int64_t ntiles = (K.N + K.bn - 1) / K.bn;
    int base = 0;
    for (int64_t t0 = 0; t0 < ntiles; t0 += 256) {
        const int64_t t = t0 + tid;
        bool keep = false;
        if (t < ntiles) {
            keep = all;
            if (!keep) {
                float xl[3], xh[3], lb = 0.0f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    xl[c] = 3.0e38f;
                    xh[c] = -3.0e38f;
                    for (int q = 0; q < per; ++q) {
                        const int64_t u = t * per + q;
                        if (u < K.nt64) {
                            xl[c] = fminf(xl[c], K.tbox[6 * u + 2 * c]);
                            xh[c] = fmaxf(xh[c], K.tbox[6 * u + 2 * c + 1]);
                        }
                    }
                    // a gap smaller than the features' rounding is treated as none
                    const float slack = 0x1p-18f * (fabsf(xl[c]) + fabsf(xh[c]) + fabsf(ylo[c]) + fabsf(yhi[c]));
                    const float gap = fmaxf(fmaxf(xl[c] - yhi[c], ylo[c] - xh[c]) - slack, 0.0f);
                    lb = fmaf(gap * gap, invW[c], lb);
                }
                keep = lb * (1.0f - 0x1p-10f) <= tmax;
                // the box bound passes: keep the tile only if some voxel's own features are
                // within its own distance bound of the draw tile's box (the same bound, per voxel)
                if (keep) {
                    keep = false;
                    float st[3];                  // the draw tile's share of the slack
#pragma unroll
                    for (int c = 0; c < 3; ++c) st[c] = 0x1p-18f * (fabsf(xl[c]) + fabsf(xh[c]));
                    // the gap bound of the draw tile's box against a (sub-)box [lo, hi] of voxel features
                    auto lower = [&](const float4& lo, const float4& hi) {
                        const float g0 = fmaxf(fmaxf(xl[0] - hi.x, lo.x - xh[0]) - st[0], 0.0f);
                        const float g1 = fmaxf(fmaxf(xl[1] - hi.y, lo.y - xh[1]) - st[1], 0.0f);
                        const float g2 = fmaxf(fmaxf(xl[2] - hi.z, lo.z - xh[2]) - st[2], 0.0f);
                        return fmaf(g2 * g2, invW[2], fmaf(g1 * g1, invW[1], g0 * g0 * invW[0])) * (1.0f - 0x1p-10f);
                    };
                    for (int b = 0; b < BM / 16 && !keep; ++b) {
                        const float4 blo = sb_lo[b];
                        if (!(lower(blo, sb_hi[b]) <= blo.w)) continue;     // no voxel of the sub-box
                        for (int v = 16 * b; v < 16 * b + 16 && !keep; ++v) {
                            const float4 lo = sv_lo[v];
                            keep = lower(lo, sv_hi[v]) <= lo.w;
                        }
                    }
                }
            }
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
        if (lane == 0) wcount[wp] = __popc(bal);
        __syncthreads();
        int pos = base, tot = 0;
        for (int q = 0; q < 8; ++q) {
            if (q < wp) pos += wcount[q];
            tot += wcount[q];
        }
        pos += __popc(bal & ((1u << lane) - 1u));
        if (keep) K.ktile[vt * K.nt64 + pos] = (int32_t)t;
        base += tot;
        __syncthreads();
    }
    if (K.order && base > 1 && base <= KEEP_SORT_MAX) {
        int n2 = 2;
        while (n2 < base) n2 <<= 1;
        int32_t* list = K.ktile + vt * K.nt64;
        float yc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) yc[c] = 0.5f * (ylo[c] + yhi[c]);
        for (int i = tid; i < n2; i += 256) {
            unsigned long long e = ~0ull;
            if (i < base) {
                const int64_t t = list[i];
                float d = 0.0f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float xl = 3.0e38f, xh = -3.0e38f;
                    for (int q = 0; q < per; ++q) {
                        const int64_t u = t * per + q;
                        if (u < K.nt64) {
                            xl = fminf(xl, K.tbox[6 * u + 2 * c]);
                            xh = fmaxf(xh, K.tbox[6 * u + 2 * c + 1]);
                        }
                    }
                    const float g = 0.5f * (xl + xh) - yc[c];
                    if (K.Wc[c] > 0.0f) d += g * g / K.Wc[c];
                }
                e = ((unsigned long long)ord_f2u(d) << 32) | (uint32_t)t;
            }
            sk[i] = e;
        }
        __syncthreads();
        // bitonic sort, ascending
        for (int len = 2; len <= n2; len <<= 1)
            for (int st = len >> 1; st > 0; st >>= 1) {
                for (int i = tid; i < n2; i += 256) {
                    const int o = i ^ st;
                    if (o > i) {
                        const bool up = (i & len) == 0;
                        const unsigned long long a = sk[i], b = sk[o];
                        if ((a > b) == up) {
                            sk[i] = b;
                            sk[o] = a;
                        }
                    }
                }
                __syncthreads();
            }
        for (int i = tid; i < base; i += 256) list[i] = (int32_t)(uint32_t)sk[i];
    }
    if (tid == 0) {
        K.kcount[vt] = base;
        if (K.tally) {      // in 64-draw units, whatever the tile width
            atomicAdd(&K.tally[0], (unsigned long long)base * per);
            atomicAdd(&K.tally[1], (unsigned long long)ntiles * per);
        }
    }
}

// ------------------------------------------------------------------ fused GEMM + filter
// One scan of a batch, as the fused kernel sees it (kernel parameter space).
struct __align__(64) ItemTc {
    CUtensorMap tmA;             // packed voxel operand, box {64, 128}
    CUtensorMap tmB;             // packed draw operand (strided for a pilot), box {64, BN}
    int64_t J, N;                // voxels; draws in this pass
    float* keys;                 // candidate lists, J x C
    int32_t* idx;
    int32_t* cnt;
    float* thr;                  // final running threshold per voxel
    const float* thr0;           // initial threshold per voxel (pilot), or null = +huge
    int ntiles, C, kt, cap;      // cap: entries a half-list keeps after a compaction (<= C2)
    int C2;                      // each voxel's list row holds two half-lists of C2 entries
    int lim;                     // a half-list is compacted once it could exceed lim entries (lim <= C2)
    int lim0;                    // ... or lim0 entries while its voxel has no finite threshold yet
    int rsel;                    // > 0: pilot that keeps the rsel smallest keys per voxel, no lists
    int hstride;                 // cnt[] / thr[] entry of half 1 of voxel j: j + hstride
    int rk;                      // top-r pilot > 0: write the rk-th smallest key (exact) instead of the r-th
    const int32_t* ktile;        // kept draw tiles per voxel tile (null: every tile)
    const int32_t* kcount;
    int64_t kstride;
    union {
        float* thr_out;          // top-r pilot: its thresholds
        const int32_t* rows;     // rescue pass: list row of each voxel position (-1: none), or null
    };
};
static_assert(sizeof(ItemTc) == 384, "ItemTc layout");

struct BatchTc {
    ItemTc item[MAX_ITEMS];
    int64_t vt_prefix[MAX_ITEMS + 1];   // voxel tiles before each item (work index space)
    int n_items;
    unsigned long long* counter;        // next work index (zeroed before the launch)
    int32_t* status;
    float* dump;                 // debug probe: raw keys, Jp x Np (null in production)
    int64_t ld_dump;
    const int32_t* dyn_count[MAX_ITEMS];   // rescue pass: voxels queued per item (null: all J)
    const int32_t* dyn_C[MAX_ITEMS];       // rescue pass: list capacity per queue position (null: the item's C)
    const int32_t* tgroup[MAX_ITEMS];      // per item: centring group of each voxel tile (null: group 0)
    int64_t grows[MAX_ITEMS];              // per item: rows of one group's copy of the draw operand
    int nseg;                    // > 1 (rescue pass): work items per voxel tile, each an interleaved
                                 // share of its draw tiles
    uint64_t wait_ns;            // bound on every barrier wait (2 s unless a test shortens it)
    int64_t withhold;            // test hook: the TMA producer never loads its draw tile of this
                                 // sequence number (< 0: off), so the waits behind it run out
};

__device__ __forceinline__ int item_of(const BatchTc& P, int64_t w) {
    int it = 0;
    while (it + 1 < P.n_items && w >= P.vt_prefix[it + 1]) ++it;
    return it;
}

// Work item w of a launch: its item, voxel tile and draw-tile segment.  With nseg > 1 (the
// rescue pass) each voxel tile is nseg work items; segment s takes the tile's kept draw tiles
// s, s + nseg, s + 2 nseg, ..., so a few voxel tiles still spread over many CTAs.
struct WorkPos {
    int it;
    int64_t vt;
    int seg, nseg;
};

__device__ __forceinline__ WorkPos decode_work(const BatchTc& P, int64_t w) {
    WorkPos r;
    r.it = item_of(P, w);
    r.nseg = P.nseg > 1 ? P.nseg : 1;
    const int64_t loc = w - P.vt_prefix[r.it];
    r.vt = loc / r.nseg;
    r.seg = (int)(loc - r.vt * r.nseg);
    return r;
}

// Bound on |computed d' - exact d'| for any draw with ||xh|| <= R.
__device__ __forceinline__ float err_bound(float cE, float ry, float R) { return cE * (2.0f * ry * R + R * R); }

// Tightens half h of voxel j's candidate list to the keys <= its kt-th key;
// returns the new threshold and updates cnt.  Each half keeps its own kt
// smallest, so the two halves together always hold the voxel's kt smallest.
__device__ __forceinline__ float compact_list(const ItemTc& I, int64_t j, int h, int& cnt, uint32_t* hist, int lane) {
    float* kj = I.keys + j * I.C + h * I.C2;
    int32_t* ij = I.idx + j * I.C + h * I.C2;
    const uint32_t T = warp_select(kj, cnt, I.kt - 1, 4, hist, lane);   // exact kt-th key
    const int q = warp_compact(kj, ij, cnt, T, I.cap, lane);
    cnt = q < I.cap ? q : I.cap;
    if (q > I.cap && lane == 0) atomicOr(&I.cnt[j + h * I.hstride], 0x40000000);   // overflow: exact scan
    return key2f(T);
}

// The fields of an item the epilogue touches per chunk, held in registers.
struct ItemRegs {
    int64_t N;
    float* keys;
    int32_t* idx;
    int C;
    int C2;                      // entries of a half-list
};

// Minimum of the 8 keys v[o .. o+7] (three-input min instructions).
__device__ __forceinline__ float min8(const float (&v)[32], int o) {
    float a, b;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(a) : "f"(v[o]), "f"(v[o + 1]), "f"(v[o + 2]));
    asm("min.f32 %0, %1, %2, %3;" : "=f"(b) : "f"(v[o + 3]), "f"(v[o + 4]), "f"(v[o + 5]));
    asm("min.f32 %0, %1, %2, %3;" : "=f"(a) : "f"(a), "f"(b), "f"(v[o + 6]));
    return fminf(a, v[o + 7]);
}

// Bits i - o of the keys v[o .. o+7] that are <= thr.
__device__ __forceinline__ uint32_t mask8(const float (&v)[32], int o, float thr) {
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) m |= (v[o + i] <= thr ? 1u : 0u) << i;
    return m;
}

// Element b (0..31, any lane-varying value) of a register array, by a select tree.
__device__ __forceinline__ float pick32(const float (&v)[32], int b) {
    float l4[16], l3[8], l2[4], l1[2];
#pragma unroll
    for (int i = 0; i < 16; ++i) l4[i] = (b & 1) ? v[2 * i + 1] : v[2 * i];
#pragma unroll
    for (int i = 0; i < 8; ++i) l3[i] = (b & 2) ? l4[2 * i + 1] : l4[2 * i];
#pragma unroll
    for (int i = 0; i < 4; ++i) l2[i] = (b & 4) ? l3[2 * i + 1] : l3[2 * i];
#pragma unroll
    for (int i = 0; i < 2; ++i) l1[i] = (b & 8) ? l2[2 * i + 1] : l2[2 * i];
    return (b & 16) ? l1[1] : l1[0];
}

// Element b (0..7, any lane-varying value) of the 8-key group v[o .. o+7], by a select tree.
__device__ __forceinline__ float pick8(const float (&v)[32], int o, int b) {
    const bool b0 = b & 1;
    const float a0 = b0 ? v[o + 1] : v[o], a1 = b0 ? v[o + 3] : v[o + 2];
    const float a2 = b0 ? v[o + 5] : v[o + 4], a3 = b0 ? v[o + 7] : v[o + 6];
    const float c0 = (b & 2) ? a1 : a0, c1 = (b & 2) ? a3 : a2;
    return (b & 4) ? c1 : c0;
}

// One 32-column chunk of the epilogue, per thread (= voxel): the minima of
// the four 8-key groups against the voxel's threshold; a thread with a passing
// group copies its 32 keys to its own row of shared memory (row_s, if any) and, group
// by passing group, appends each passing key to its half-list (starting at entry
// lbase), read back by position from the row or picked from the group's eight
// registers.  Threads never wait for one another.
// acnt != null (rescue pass): several CTAs append to the voxel's half-list, each chunk
// reserving its entries by an atomic add on the list's count; a list that would pass its
// capacity is flagged (0x40000000) instead, and its voxel takes the exact scan.
__device__ __forceinline__ void epilogue_chunk(const ItemRegs& I, float (&v)[32], int64_t n0, int64_t lbase, float thr,
                                               int& cnt, float* row_s, int* acnt) {
    if (n0 + 32 > I.N) {
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (n0 + i >= I.N) v[i] = __int_as_float(0x7F800000);   // +inf: never kept
    }
    const float g0 = min8(v, 0), g1 = min8(v, 8), g2 = min8(v, 16), g3 = min8(v, 24);
    float gm;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(gm) : "f"(g0), "f"(g1), "f"(g2));
    if (fminf(gm, g3) > thr) return;
    // the passing keys are read back by position from this thread's own row of shared memory,
    // or (row_s null: passing keys are rare) picked from the registers by a select tree
    if (row_s) {
        float4* dst = (float4*)row_s;
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    if (!acnt) {
        // only the 8-key groups whose minimum passes are examined key by key, in key order
        float* kp = I.keys + lbase;
        int32_t* ip = I.idx + lbase;
        const float gmin[4] = {g0, g1, g2, g3};
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            if (gmin[g] > thr) continue;
            uint32_t m = mask8(v, 8 * g, thr);
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                kp[cnt] = row_s ? row_s[8 * g + b] : pick8(v, 8 * g, b);
                ip[cnt] = (int32_t)(n0 + 8 * g + b);
                ++cnt;
            }
        }
        return;
    }
    uint32_t m = 0;
    if (g0 <= thr) m |= mask8(v, 0, thr);
    if (g1 <= thr) m |= mask8(v, 8, thr) << 8;
    if (g2 <= thr) m |= mask8(v, 16, thr) << 16;
    if (g3 <= thr) m |= mask8(v, 24, thr) << 24;
    {
        const int n = __popc(m);
        int pos = atomicAdd(acnt, n);
        if (pos + n > I.C2) {
            atomicOr(acnt, 0x40000000);
            return;
        }
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            I.keys[lbase + pos] = (row_s ? row_s[b] : pick32(v, b));
            I.idx[lbase + pos] = (int32_t)(n0 + b);
            ++pos;
        }
    }
}


// Per-thread state of a top-r pilot: the voxel's kept keys A[i * 128] (i < n_in), a
// max-heap once filled (A[0] the largest), its maximum amax once n_in = r, and the
// quick-reject threshold thr = min(thr_in, amax) (thr_in alone until r keys are in).
// Each thread owns one column of the shared array, so heap moves of different lanes
// never share a bank.
struct TopR {
    float* A;
    int r, n_in;
    float amax, thr_in, thr;
};

// Adds key x to a top-r set: while filling, a sift-up insert; once full, x replaces the
// root (the largest key) if it is smaller, and sifts down.  The kept multiset is the same
// as any other exact top-r bookkeeping's.
__device__ __forceinline__ void topr_add(TopR& S, float x) {
    if (S.n_in < S.r) {
        int i = S.n_in++;
        while (i > 0) {
            const int p = (i - 1) >> 1;
            const float ap = S.A[p * 128];
            if (ap >= x) break;
            S.A[i * 128] = ap;
            i = p;
        }
        S.A[i * 128] = x;
        if (S.n_in == S.r) {
            S.amax = S.A[0];
            S.thr = fminf(S.thr_in, S.amax);
        }
    } else if (x < S.amax) {
        int i = 0;
        for (;;) {
            int c = 2 * i + 1;
            if (c >= S.r) break;
            float ac = S.A[c * 128];
            if (c + 1 < S.r) {
                const float a2 = S.A[(c + 1) * 128];
                if (a2 > ac) {
                    ac = a2;
                    ++c;
                }
            }
            if (ac <= x) break;
            S.A[i * 128] = ac;
            i = c;
        }
        S.A[i * 128] = x;
        S.amax = S.A[0];
        S.thr = fminf(S.thr_in, S.amax);
    }
}

// One 32-column chunk of a top-r pilot: keys <= thr join the kept set (the
// largest kept key leaves once r are kept), so the set ends as the r smallest
// keys that are <= thr_in.  Rare after the first tiles.
__device__ __forceinline__ void topr_chunk(TopR& S, float (&v)[32], int64_t n0, int64_t N) {
    if (n0 + 32 > N) {
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (n0 + i >= N) v[i] = __int_as_float(0x7F800000);
    }
    const float g0 = min8(v, 0), g1 = min8(v, 8), g2 = min8(v, 16), g3 = min8(v, 24);
    float gm;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(gm) : "f"(g0), "f"(g1), "f"(g2));
    if (fminf(gm, g3) > S.thr) return;
    // group by group (a later group's mask is taken against the threshold as it then stands,
    // which keeps the same keys as one mask taken first)
    const float gmin[4] = {g0, g1, g2, g3};
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        if (gmin[g] > S.thr) continue;
        uint32_t m = mask8(v, 8 * g, S.thr);
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            topr_add(S, pick8(v, 8 * g, b));
        }
    }
}

// The rk-th smallest (1-based) of the n keys col[i * 128], i < n (rk <= n).
__device__ __forceinline__ float kth_of_column(const float* col, int n, int rk) {
    float out = 3.0e38f;
    for (int i = 0; i < n; ++i) {
        const float v = col[i * 128];
        int lt = 0, eq = 0;
        for (int q = 0; q < n; ++q) {
            const float u = col[q * 128];
            lt += u < v;
            eq += u == v;
        }
        if (lt < rk && rk <= lt + eq) out = v;
    }
    return out;
}

// Persistent fused kernel over the (scan, 128-voxel tile) work items of a batch,
// handed out round-robin in the order of the work index space (costliest
// scans first).  All roles walk the same sequence; the shared-memory ring and
// the TMEM accumulators keep their phases across items.
template <int NKB, int STAGES, int BN, bool DUMP, bool TOPR>
__global__ void __launch_bounds__(tc_threads(TOPR, BN), tc_epi_warps(TOPR, BN) == 8 ? 2 : 3)
    k_tc_topk(const __grid_constant__ BatchTc P) {
    constexpr int B_KBLK_BYTES = BN * KBLK * 2;
    constexpr int EPI = tc_epi_warps(TOPR, BN);                  // epilogue warps
    constexpr int CSTEP = EPI / 4;                               // chunk stride of an epilogue warp
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                                          // NKB x 16 KB
    uint8_t* sB = smem + NKB * A_KBLK_BYTES;                     // STAGES x NKB x BN rows
    constexpr int ROW_FLOATS = tc_rows(NKB, TOPR) ? 32 * EPI * ROW_LD : 0;
    float* sRow = (float*)(sB + STAGES * NKB * B_KBLK_BYTES);         // 32 EPI threads x ROW_LD (if any)
    uint32_t* hist = (uint32_t*)(sRow + ROW_FLOATS);                    // EPI warps x 256
    uint64_t* bars = (uint64_t*)(hist + EPI * 256);
    uint64_t* full = bars;                  // [STAGES]
    uint64_t* empty = bars + STAGES;        // [STAGES]
    uint64_t* tfull = bars + 2 * STAGES;    // [2]
    uint64_t* tempty = bars + 2 * STAGES + 2;
    uint64_t* afull = bars + 2 * STAGES + 4;
    uint64_t* aempty = bars + 2 * STAGES + 5;
    uint64_t* ifull = bars + 2 * STAGES + 6;    // [2] work-item mailbox
    uint64_t* iempty = bars + 2 * STAGES + 8;   // [2]
    volatile long long* slot = (volatile long long*)(bars + 2 * STAGES + 10);   // [2]
    uint32_t* tmem_holder = (uint32_t*)(bars + 2 * STAGES + 12);
    volatile int* s_err = (volatile int*)(tmem_holder + 1);
    uint64_t* drain = bars + 2 * STAGES + 13;   // MMA thread: all of its MMAs complete

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t total = P.vt_prefix[P.n_items];
    const uint64_t WAIT_NS = P.wait_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(ptx::smem_u32(&full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(ptx::smem_u32(&tfull[a]), 1);
            ptx::mbar_init(ptx::smem_u32(&tempty[a]), EPI);
        }
        ptx::mbar_init(ptx::smem_u32(afull), 1);
        ptx::mbar_init(ptx::smem_u32(aempty), 1);
        ptx::mbar_init(ptx::smem_u32(drain), 1);
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(ptx::smem_u32(&ifull[a]), 1);
            ptx::mbar_init(ptx::smem_u32(&iempty[a]), 1 + EPI);   // MMA thread + the epilogue warps
        }
        *s_err = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(tmem_holder), 2 * BN);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            uint32_t gt = 0;
            // loads this thread issued and has not seen land: per ring stage the parity of the
            // phase it last loaded, and the A tile's; waited for before the CTA exits, so no
            // copy into this CTA's shared memory is still in flight after a bounded wait ran out
            uint32_t st_issued = 0, st_parity = 0, a_issued = 0, a_parity = 0;
            for (uint32_t ic = 0;; ++ic) {
                // take the next work item and post it to the other roles (a rescue item's voxel
                // tiles past its queued voxels are skipped)
                long long w = (long long)atomicAdd(P.counter, 1ull);
                while (w < total && !*s_err) {
                    const WorkPos wp = decode_work(P, w);
                    const int32_t* dc = P.dyn_count[wp.it];
                    if (!dc || wp.vt * BM < (long long)*dc) break;
                    w = (long long)atomicAdd(P.counter, 1ull);
                }
                if (w >= total || *s_err) w = -1;
                const uint32_t sl = ic & 1u;
                if (!ptx::mbar_wait(ptx::smem_u32(&iempty[sl]), ((ic >> 1) & 1u) ^ 1u, WAIT_NS)) { *s_err = 1; w = -1; }
                slot[sl] = w;
                ptx::mbar_arrive(ptx::smem_u32(&ifull[sl]));
                if (w < 0) break;
                const WorkPos wp = decode_work(P, w);
                const ItemTc& I = P.item[wp.it];
                const int64_t vt = wp.vt;
                const int64_t m0 = vt * BM;
                const int ntiles = I.ktile ? I.kcount[vt] : I.ntiles;
                const int32_t* kt_list = I.ktile ? I.ktile + vt * I.kstride : nullptr;
                const int64_t gofs = P.tgroup[wp.it] ? (int64_t)P.tgroup[wp.it][vt] * P.grows[wp.it] : 0;   // the group's B copy
                ptx::tma_prefetch_desc(&I.tmA);
                ptx::tma_prefetch_desc(&I.tmB);
                // the previous item's MMAs must be done with the A tile
                if (!ptx::mbar_wait(ptx::smem_u32(aempty), (ic & 1u) ^ 1u, WAIT_NS)) { *s_err = 1; break; }
                const uint32_t ab = ptx::smem_u32(afull);
                ptx::mbar_arrive_expect_tx(ab, NKB * A_KBLK_BYTES);
                for (int kb = 0; kb < NKB; ++kb)
                    ptx::tma_load_2d(ptx::smem_u32(sA + kb * A_KBLK_BYTES), &I.tmA, ab, kb * KBLK, (int32_t)m0);
                a_issued = 1;
                a_parity = ic & 1u;
                for (int t = wp.seg; t < ntiles; t += wp.nseg, ++gt) {
                    const uint32_t s = gt % STAGES;
                    const uint32_t ph = (gt / STAGES) & 1u;
                    if (!ptx::mbar_wait(ptx::smem_u32(&empty[s]), ph ^ 1u, WAIT_NS)) { *s_err = 1; break; }
                    if (*s_err) break;
                    if ((int64_t)gt == P.withhold) continue;   // test hook: this stage never fills
                    const uint32_t fb = ptx::smem_u32(&full[s]);
                    ptx::mbar_arrive_expect_tx(fb, NKB * B_KBLK_BYTES);
                    for (int kb = 0; kb < NKB; ++kb)
                        ptx::tma_load_2d(ptx::smem_u32(sB + (s * NKB + kb) * B_KBLK_BYTES), &I.tmB, fb, kb * KBLK,
                                         (int32_t)((kt_list ? kt_list[t] : t) * BN + gofs));
                    st_issued |= 1u << s;
                    st_parity = (st_parity & ~(1u << s)) | (ph << s);
                }
            }
            for (int s = 0; s < STAGES; ++s)
                if ((st_issued >> s) & 1u)
                    if (!ptx::mbar_wait(ptx::smem_u32(&full[s]), (st_parity >> s) & 1u, WAIT_NS)) *s_err = 1;
            if (a_issued && !ptx::mbar_wait(ptx::smem_u32(afull), a_parity, WAIT_NS)) *s_err = 1;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (single thread)
        if (lane == 0) {
            constexpr uint32_t idesc = ptx::idesc_bf16_f32(BM, BN);
            const uint32_t a_base = ptx::smem_u32(sA);
            uint32_t gt = 0;
            for (uint32_t ic = 0;; ++ic) {
                const uint32_t sl = ic & 1u;
                long long w = -1;
                if (ptx::mbar_wait(ptx::smem_u32(&ifull[sl]), (ic >> 1) & 1u, WAIT_NS)) w = slot[sl];
                else *s_err = 1;
                ptx::mbar_arrive(ptx::smem_u32(&iempty[sl]));
                if (w < 0) break;
                const WorkPos wp = decode_work(P, w);
                const ItemTc& IM = P.item[wp.it];
                const int ntiles = IM.ktile ? IM.kcount[wp.vt] : IM.ntiles;
                if (!ptx::mbar_wait(ptx::smem_u32(afull), ic & 1u, WAIT_NS)) { *s_err = 1; break; }
                for (int t = wp.seg; t < ntiles; t += wp.nseg, ++gt) {
                    const uint32_t s = gt % STAGES;
                    const uint32_t ph = (gt / STAGES) & 1u;
                    const uint32_t acc = gt & 1u;
                    const uint32_t aph = (gt >> 1) & 1u;
                    if (*s_err) break;
                    if (!ptx::mbar_wait(ptx::smem_u32(&tempty[acc]), aph ^ 1u, WAIT_NS) ||
                        !ptx::mbar_wait(ptx::smem_u32(&full[s]), ph, WAIT_NS)) {
                        *s_err = 1;
                        break;
                    }
                    if (*s_err) break;
                    ptx::tc_fence_after();
                    const uint32_t d_tmem = tmem + acc * BN;
                    const uint32_t b_base = ptx::smem_u32(sB + s * NKB * B_KBLK_BYTES);
#pragma unroll
                    for (int kb = 0; kb < NKB; ++kb) {
#pragma unroll
                        for (int kk = 0; kk < KBLK / 16; ++kk) {
                            const uint64_t ad = ptx::desc_sw128(a_base + kb * A_KBLK_BYTES + kk * 32);
                            const uint64_t bd = ptx::desc_sw128(b_base + kb * B_KBLK_BYTES + kk * 32);
                            ptx::mma_bf16(d_tmem, ad, bd, idesc, (kb | kk) ? 1u : 0u);
                        }
                    }
                    ptx::mma_commit(ptx::smem_u32(&empty[s]));
                    ptx::mma_commit(ptx::smem_u32(&tfull[acc]));
                }
                ptx::mma_commit(ptx::smem_u32(aempty));   // A tile free once these MMAs complete
            }
            // every MMA this thread issued has completed before TMEM is freed, also when a
            // bounded wait ran out and no epilogue waited for the last accumulators
            ptx::mma_commit(ptx::smem_u32(drain));
            if (!ptx::mbar_wait(ptx::smem_u32(drain), 0u, WAIT_NS)) *s_err = 1;
        }
    } else {
        // ---------------- epilogue: warps 2 .. 2 + EPI - 1, thread <-> voxel
        const int q = warp & 3;                          // TMEM lane quadrant of this warp
        const int hh = EPI == 8 ? (warp - 2) >> 2 : 0;   // chunk parity and half-list (0 with 4 warps)
        const int row = q * 32 + lane;
        uint32_t* whist = hist + (warp - 2) * 256;
        float* row_s = tc_rows(NKB, TOPR) ? sRow + (threadIdx.x - 64) * ROW_LD : nullptr;
        uint32_t gt = 0;
        bool stop = false;
        for (uint32_t ic = 0; !stop; ++ic) {
            const uint32_t sl = ic & 1u;
            long long w = -1;
            if (ptx::mbar_wait(ptx::smem_u32(&ifull[sl]), (ic >> 1) & 1u, WAIT_NS)) w = slot[sl];
            else *s_err = 1;
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&iempty[sl]));
            if (w < 0) break;
            const WorkPos wp = decode_work(P, w);
            const ItemTc& I = P.item[wp.it];
            // list capacity (a rescue pass reads the one its layout kernel chose) and half-list size
            const int Cl = P.dyn_C[wp.it] ? *P.dyn_C[wp.it] : I.C;
            const int C2l = P.dyn_C[wp.it] ? (I.C2 == I.C ? Cl : Cl / 2) : I.C2;
            const ItemRegs R{I.N, I.keys, I.idx, Cl, C2l};
            const int64_t vt = wp.vt;
            const int ntiles = I.ktile ? I.kcount[vt] : I.ntiles, lim = I.lim, lim0 = I.lim0;
            const int32_t* kt_list = I.ktile ? I.ktile + vt * I.kstride : nullptr;
            const int64_t m0 = vt * BM;
            const int64_t jbase = m0 + q * 32;
            const int64_t j = jbase + lane;
            // the voxel's list row; a rescue pass lists by queue position (rows[] maps positions
            // to the packed rows of queued voxels, -1 for padding)
            const int64_t jrow = (!TOPR && I.rows) ? (j < I.J && I.rows[j] >= 0 ? j : -1) : j;
            const bool valid = j < I.J && jrow >= 0;
            float thr = valid ? (I.thr0 ? I.thr0[j] : 3.0e38f) : -3.0e38f;
            int cnt = 0;
            const int64_t lbase = jrow * (int64_t)Cl + hh * C2l;     // this thread's half-list
            // rescue pass: the voxel's threshold is fixed and its draw tiles are shared among
            // several CTAs, which reserve list entries atomically (no compaction)
            const bool shared_list = !TOPR && I.rows != nullptr;
            int* acnt = (shared_list && valid) ? &I.cnt[jrow + hh * I.hstride] : nullptr;
            TopR S{sRow + (threadIdx.x - 64), TOPR ? I.rsel : 0, 0, -3.0e38f, thr, thr};
            // the next tile's draw offset is loaded a tile ahead, off the path from the
            // accumulator's arrival to its first use
            int tnext = kt_list && ntiles > wp.seg ? kt_list[wp.seg] : 0;
            for (int t = wp.seg; t < ntiles; t += wp.nseg, ++gt) {
                const int64_t nbase = (int64_t)(kt_list ? tnext : t) * BN;
                if (kt_list && t + wp.nseg < ntiles) tnext = kt_list[t + wp.nseg];
                const uint32_t acc = gt & 1u;
                const uint32_t aph = (gt >> 1) & 1u;
                // one vote per tile: this warp's wait ran out, or another role flagged an error
                // (a role that stopped leaves this wait to run out at its bound)
                {
                    const bool ok = ptx::mbar_wait(ptx::smem_u32(&tfull[acc]), aph, WAIT_NS);
                    if (!ok) *s_err = 1;
                    if (__any_sync(0xFFFFFFFFu, !ok || *s_err != 0)) { stop = true; break; }
                }
                ptx::tc_fence_after();
                const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + acc * BN;
                if (DUMP) {
                    for (int c = hh; c < BN / 32; c += CSTEP) {
                        uint32_t r[32];
                        ptx::tmem_ld32_async(ta + c * 32, r);
                        ptx::tmem_wait_ld();
                        ptx::tmem_fence_regs(r);
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            P.dump[(m0 + row) * P.ld_dump + nbase + c * 32 + i] = __uint_as_float(r[i]);
                    }
                } else {
                    // one 32-column load at a time (fewer live registers than overlapping two
                    // loads, which measured slower); the chunk loop unrolled
#pragma unroll
                    for (int c = hh; c < BN / 32; c += CSTEP) {
                        uint32_t r[32];
                        ptx::tmem_ld32_async(ta + c * 32, r);
                        ptx::tmem_wait_ld();
                        ptx::tmem_fence_regs(r);
                        float v[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
                        // a lane without a voxel (padding rows) keeps nothing, whatever its keys
                        if (valid) {
                            if constexpr (TOPR) topr_chunk(S, v, nbase + c * 32, R.N);
                            else epilogue_chunk(R, v, nbase + c * 32, lbase, thr, cnt, row_s, acnt);
                        }
                    }
                }
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&tempty[acc]));
                if (DUMP || TOPR || shared_list) continue;
                // compaction of lists that might not fit the next tile
                // a list without a threshold yet (the coarsest pilot) is first cut early, at
                // lim0: from then on far fewer keys pass than the everything of a +inf start
                uint32_t need = __ballot_sync(0xFFFFFFFFu, valid && cnt > (thr >= 3.0e38f ? lim0 : lim) - BN / CSTEP);
                while (need) {
                    const int src = __ffs(need) - 1;
                    need &= need - 1;
                    int c2 = __shfl_sync(0xFFFFFFFFu, cnt, src);
                    const float nt = compact_list(I, __shfl_sync(0xFFFFFFFFu, jrow, src), hh, c2, whist, lane);
                    if (lane == src) {
                        cnt = c2;
                        thr = nt;
                    }
                }
            }
            if (valid && !DUMP && !stop) {
                if (TOPR) {
                    // the r-th smallest key, rounded up to its 24-bit prefix (as the list
                    // pilots' three-digit selection gives it), or none; a finest split-form
                    // pilot writes its rk-th smallest key (turned into a need threshold next)
                    const float t = I.rk > 0 ? (S.n_in >= I.rk ? kth_of_column(S.A, S.n_in, I.rk) : 3.0e38f)
                                             : (S.n_in == S.r ? key2f(f2key(S.amax) | 0xFFu) : 3.0e38f);
                    I.thr_out[j] = t;
                    if (t >= 3.0e38f) atomicAdd(&P.status[7], 1);
                } else {
                    // cnt[] was zeroed (a shared list counted its entries as they were reserved);
                    // keeps the overflow bit
                    if (!shared_list) atomicOr(&I.cnt[jrow + hh * I.hstride], cnt);
                    I.thr[jrow + hh * I.hstride] = thr;
                    if (EPI == 4) I.thr[jrow + I.hstride] = 3.0e38f;   // the unused half-list bounds nothing
                }
            }
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 2 * BN);
    }
    if (threadIdx.x == 0 && *s_err) atomicExch(&P.status[0], ABC_ERR_TIMEOUT);
}

// Pilot threshold: the r-th smallest key of each voxel's pilot list, then the
// list is emptied for the next pass.
struct PilotItem {
    float* keys;
    int32_t* cnt;
    float* thr0;
    int64_t J;
    int C, r;
    int C2;
    int64_t hstride;
};

// Moves half-list 1 of a list row (entries [C2, C2 + c1)) to follow half-list 0
// (entries [0, c0)), keys and (when given) draw indices, four rows of 32 at a time with
// their loads in flight together.  A batch is read before it is written, and every write
// lands below the next batch's reads (c0 <= C2), so the copy is safe in place.
__device__ __forceinline__ void merge_halves(float* kj, int32_t* ij, int C2, int c0, int c1, int lane) {
    if (c0 == C2 || c1 == 0) return;
    constexpr int RA = 4;
    for (int base = 0; base < c1; base += 32 * RA) {
        float k[RA];
        int32_t id[RA];
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const int i = base + 32 * r + lane;
            k[r] = i < c1 ? kj[C2 + i] : 0.0f;
            id[r] = (ij && i < c1) ? ij[C2 + i] : 0;
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const int i = base + 32 * r + lane;
            if (i < c1) {
                kj[c0 + i] = k[r];
                if (ij) ij[c0 + i] = id[r];
            }
        }
    }
    __syncwarp();
}

struct BatchPilot {
    PilotItem item[MAX_ITEMS];
    int64_t v_prefix[MAX_ITEMS + 1];
    int n_items;
    int32_t* status;
};

__global__ void k_pilot_threshold(const __grid_constant__ BatchPilot B) {
    __shared__ uint32_t hist[8][256];
    __shared__ float gbuf[8][256];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * 8 + wid;
    if (g >= B.v_prefix[B.n_items]) return;
    int it = 0;
    while (it + 1 < B.n_items && g >= B.v_prefix[it + 1]) ++it;
    const PilotItem& I = B.item[it];
    const int64_t j = g - B.v_prefix[it];
    const int raw0 = I.cnt[j], raw1 = I.cnt[j + I.hstride];
    const int c0 = raw0 & 0x3FFFFFFF, c1 = raw1 & 0x3FFFFFFF, c = c0 + c1;
    float t = 3.0e38f;
    // the r-th smallest key of the two half-lists, rounded up to its 24-bit prefix
    if (!((raw0 | raw1) & 0x40000000) && c >= I.r) {
        float* kj = I.keys + j * I.C;
        merge_halves(kj, nullptr, I.C2, c0, c1, lane);
        t = key2f(warp_select_exact(kj, c, I.r - 1, hist[wid], gbuf[wid], 256, lane).K | 0xFFu);
    }
    if (lane == 0) {
        I.thr0[j] = t;
        I.cnt[j] = 0;
        I.cnt[j + I.hstride] = 0;
        if (t >= 3.0e38f) atomicAdd(&B.status[7], 1);     // diagnostics: pilot level without a threshold
    }
}

// Split form, after the finest pilot: the pilot key K of rank rk (four standard deviations
// above the rank of the k-th draw) gives the distance estimate K + ||yh||^2 - c0, and the
// main pass keeps every draw with key <= need_key(that estimate).  This covers the
// finalize's net in all but a small fraction of voxels (measured: under 1 %), which its
// certificate detects and the rescue pass resolves; bounding the estimate once more
// (dist_ub) would cover them all at about twice the list length.
struct NeedItem {
    float* thr0;
    const float* ynorm;
    const float* c0;
    const float* dn;
    int64_t J;
    SplitCoef sc;
};

struct BatchNeed {
    NeedItem item[MAX_ITEMS];
    int64_t v_prefix[MAX_ITEMS + 1];
    int n_items;
};

__global__ void k_need_threshold(const __grid_constant__ BatchNeed B) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= B.v_prefix[B.n_items]) return;
    int it = 0;
    while (it + 1 < B.n_items && g >= B.v_prefix[it + 1]) ++it;
    const NeedItem& I = B.item[it];
    const int64_t j = g - B.v_prefix[it];
    const float K = I.thr0[j];
    if (!(K < 1.0e30f)) return;          // no pilot threshold: the main pass starts without one
    const float yn = I.ynorm[j], c0 = I.c0[j], dn = I.dn[j];
    I.thr0[j] = need_key(fmaxf(K + yn - c0, 0.0f), yn, c0, dn, I.sc);
}

// Rescue pass set-up (split form).  The first finalize queued voxels in arrival order
// (qrows, qthr, qdk, at most cap of them).  A rescued voxel tile must lie in one centring
// group, so the queue is sorted by group into runs padded to whole tiles: per group its
// count, then each group's first position, then the placement, which also copies the
// voxel's packed operand row into the compact A operand.  The rescue pass lists by queue
// position (counts and thresholds of its own, zeroed on the host).
// Queue words: [0] voxels queued, [1] positions in use (runs padded), [2, 2+G) counts,
// [2+G, 2+2G) cursors, [2+2G, 3+3G) first positions, [3+3G] the rescue lists' capacity.
struct RescueItem {
    int32_t* words;
    const int32_t* qrows;
    const float* qthr;
    const float* qdk;
    int32_t* rows;               // sorted by group (-1: padding)
    float* thr;
    float* dk;
    int32_t* rtg;                // group of each rescue tile
    int64_t cap, Jg, J;          // cap: the queue capacity the first finalize used
    int G, Kp;
    const __nv_bfloat16* A;
    __nv_bfloat16* RA;
    int64_t list_entries;        // the scan's candidate-list space (entries), shared by the rescue lists
    int Cr;                      // the rescue lists' capacity with the whole queue in use
};

struct BatchRescue {
    RescueItem item[MAX_ITEMS];
    int n_items;
};

__device__ __forceinline__ int64_t rescue_queued(const RescueItem& I) {
    const int64_t c = I.words[0];
    return c < I.cap ? c : I.cap;
}

__global__ void k_rescue_count(const __grid_constant__ BatchRescue B) {
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    for (int it = 0; it < B.n_items; ++it) {
        const RescueItem& I = B.item[it];
        const int64_t n = rescue_queued(I);
        for (int64_t p = t0; p < n; p += nt) {
            const int32_t row = I.qrows[p];
            if (row >= 0 && row < I.J) atomicAdd(&I.words[2 + row / I.Jg], 1);
        }
    }
}

// one block per item
__global__ void k_rescue_layout(const __grid_constant__ BatchRescue B) {
    const RescueItem& I = B.item[blockIdx.x];
    int32_t* cnt_g = I.words + 2;
    int32_t* cur_g = I.words + 2 + I.G;
    int32_t* first = I.words + 2 + 2 * I.G;
    if (threadIdx.x == 0) {
        int32_t off = 0;
        for (int g = 0; g < I.G; ++g) {
            first[g] = off;
            cur_g[g] = off;
            off += (cnt_g[g] + BM - 1) / BM * BM;
        }
        first[I.G] = off;
        I.words[1] = off;
        // the list space over the positions in use: a short queue gets long lists (at most 2^26
        // entries, so that a list's count stays far below its overflow flag, bit 30)
        int64_t cap = I.list_entries / (off > 0 ? off : 1);
        cap = cap < (1 << 26) ? cap : (1 << 26);
        cap &= ~(int64_t)1;
        I.words[2 + 3 * I.G + 1] = (int32_t)(cap > I.Cr ? cap : I.Cr);
    }
    __syncthreads();
    const int32_t total = I.words[1];
    for (int32_t t = threadIdx.x; t < total / BM; t += blockDim.x) {
        int g = 0;
        while (g + 1 < I.G && first[g + 1] <= t * BM) ++g;
        I.rtg[t] = g;
    }
    // padding positions of each run: no voxel, an all-zero operand row
    for (int g = 0; g < I.G; ++g)
        for (int32_t p = first[g] + cnt_g[g] + (int32_t)threadIdx.x; p < first[g + 1]; p += blockDim.x) {
            I.rows[p] = -1;
            uint4* dst = (uint4*)(I.RA + (int64_t)p * I.Kp);
            for (int q = 0; q < I.Kp / 8; ++q) dst[q] = make_uint4(0u, 0u, 0u, 0u);
        }
}

// one warp per queued voxel
__global__ void k_rescue_place(const __grid_constant__ BatchRescue B) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int it = 0; it < B.n_items; ++it) {
        const RescueItem& I = B.item[it];
        const int64_t n = rescue_queued(I);
        for (int64_t p = w0; p < n; p += nw) {
            const int64_t row = I.qrows[p];
            if (row < 0 || row >= I.J) continue;      // (never written by the finalize: skipped as by the count)
            int pos = 0;
            if (lane == 0) pos = atomicAdd(&I.words[2 + I.G + row / I.Jg], 1);
            pos = __shfl_sync(0xFFFFFFFFu, pos, 0);
            const uint4* src = (const uint4*)(I.A + row * I.Kp);
            uint4* dst = (uint4*)(I.RA + (int64_t)pos * I.Kp);
            for (int q = lane; q < I.Kp / 8; q += 32) dst[q] = src[q];
            if (lane == 0) {
                I.rows[pos] = (int32_t)row;
                I.thr[pos] = I.qthr[p];
                I.dk[pos] = I.qdk[p];
            }
        }
    }
}

// ------------------------------------------------------------------ finalize
struct FinItem {
    int64_t J, N;
    int L, k, C, kt, mode, sortcap;
    int C2;                      // the list row's two half-lists start at 0 and C2
    int64_t hstride;             // cnt[] / thr[] of half 1: list row + hstride
    float cacc;                  // (3 Kp + L + 16) 2^-24: the keys' fp32 accumulation (both certificates)
    int ldy, ldx;
    const float* y;
    const float* x;
    const float* ynorm;          // per packed voxel row
    const float* c0;             // split form: -2 delta . yh per packed voxel row
    const float* dn;             // split form: ||delta|| per packed voxel row
    const int32_t* perm;         // packed voxel row -> voxel (null: identity)
    const int32_t* xperm;        // packed draw row -> draw (null: identity)
    const float* xs;             // draws in packed order, fp32 (row stride ldxs)
    int ldxs;
    const float* tbox;           // 64-draw tile feature boxes (null: draws not ordered)
    const float* fy;             // voxel segment features per packed voxel row
    int64_t nt64;
    float Wc[3];
    float* keys;
    int32_t* idx;
    int32_t* cnt;
    const float* thr;
    int32_t* out_idx;
    float* out_dist;
    const float* w;              // frame weights (device copy in the workspace)
    const int32_t* rows;         // rescue pass: packed row of each queue position (lists by position), or null
    const int32_t* rcount;       // rescue pass: voxels queued
    const int32_t* dyn_C;        // rescue pass: list capacity per queue position (null: C)
    int32_t* rq_rows;            // first pass of the split form: the rescue queue (null: no rescue)
    float* rq_thr;
    float* rq_dk;                // the queued net's exact k-th distance (first pass writes, rescue reads)
    int32_t* rq_count;
    int64_t rq_cap;
};

struct BatchFin {
    FinItem item[MAX_ITEMS];
    int64_t v_prefix[MAX_ITEMS + 1];
    int n_items;
    int sortcap;                 // largest sortcap of the batch (shared-memory sizing)
    int32_t* status;
    int force_rescue;            // test hook bits: 1 no first net is certified, 2 no rescue net is
};

// Exact fp32 distance sum_l w_l (y_l - x_l)^2 of a draw row in one fixed
// order: 4-frame partial sums p_h (frames 4h..4h+3 in order), combined by the
// pairing tree p_h + p_{h+o}, o = G/2 .. 1 (G = the power of two covering L
// in 4-frame pieces).  group_dist_n evaluates it with G lanes per row (one
// 16-byte load per lane, a butterfly over the group), lane_dist with one lane
// per row; both give the same value for a (voxel, draw) pair.  y and w live in
// shared memory.
__device__ __forceinline__ float lane_dist(const float* ys, const float* ws, const float* xrow, int L, int G) {
    float p[16];
    const float4* xr = (const float4*)xrow;
#pragma unroll
    for (int h = 0; h < 16; ++h) {
        p[h] = 0.0f;
        const int l = 4 * h;
        if (h < G && l < L) {
            const float4 v = __ldg(xr + h);
            const float xv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (l + q < L) {
                    const float e = ys[l + q] - xv[q];
                    p[h] = fmaf(ws[l + q] * e, e, p[h]);
                }
        }
    }
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1)
        if (o < G) {
#pragma unroll
            for (int h = 0; h < o; ++h) p[h] += p[h + o];
        }
    return p[0];
}

// NR rows per group of G lanes, all loads issued before the arithmetic; the
// lane's four frames 4h..4h+3 of y and w come in registers (yq, wq; zero
// weight past L).  Every lane of the warp must call it (full-warp shuffles).
template <int NR>
__device__ __forceinline__ void group_dist_n(const float (&yq)[4], const float (&wq)[4], const float* const (&xr)[NR],
                                             int L, int h, int G, float (&d)[NR]) {
    const int l = 4 * h;
    float4 v[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        d[r] = 0.0f;
        if (l < L) v[r] = __ldg((const float4*)xr[r] + h);
    }
    if (l < L) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const float xv[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (l + q < L) {
                    const float e = yq[q] - xv[q];
                    d[r] = fmaf(wq[q] * e, e, d[r]);
                }
        }
    }
    for (int o = G >> 1; o > 0; o >>= 1) {
#pragma unroll
        for (int r = 0; r < NR; ++r) d[r] += __shfl_xor_sync(0xFFFFFFFFu, d[r], o);
    }
}

// The lane's four frames 4h..4h+3 of four draw rows (unloaded past L), issued together.
__device__ __forceinline__ void load_rows4(const float* const (&xr)[4], int L, int h, float4 (&v)[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
        if (4 * h < L) v[r] = __ldg((const float4*)xr[r] + h);
}

// Four rows per group of G >= 4 lanes, as group_dist_n, but the butterfly is a
// reduce-scatter: the first level keeps two of the four rows per lane, the second
// one, the rest sum that one; each addition pairs the same operands as the full
// butterfly, so every row's value is the same.  Lanes h with h % (G / 4) == 0
// return row 2 [h & G/2] + [h & G/4].  v: the rows' frames from load_rows4.
__device__ __forceinline__ float group_dist_scatter4_v(const float (&yq)[4], const float (&wq)[4], const float4 (&v)[4],
                                                       int L, int h, int G, int& row) {
    const int l = 4 * h;
    float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (l < L) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float xv[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (l + q < L) {
                    const float e = yq[q] - xv[q];
                    d[r] = fmaf(wq[q] * e, e, d[r]);
                }
        }
    }
    const int o1 = G >> 1, o2 = G >> 2;
    const bool b1 = (h & o1) != 0, b2 = (h & o2) != 0;
    const float s0 = b1 ? d[0] : d[2], s1 = b1 ? d[1] : d[3];
    const float x0 = (b1 ? d[2] : d[0]) + __shfl_xor_sync(0xFFFFFFFFu, s0, o1);
    const float x1 = (b1 ? d[3] : d[1]) + __shfl_xor_sync(0xFFFFFFFFu, s1, o1);
    float y = (b2 ? x1 : x0) + __shfl_xor_sync(0xFFFFFFFFu, b2 ? x0 : x1, o2);
    for (int o = o2 >> 1; o > 0; o >>= 1) y += __shfl_xor_sync(0xFFFFFFFFu, y, o);
    row = (b1 ? 2 : 0) + (b2 ? 1 : 0);
    return y;
}

__device__ __forceinline__ float group_dist_scatter4(const float (&yq)[4], const float (&wq)[4],
                                                     const float* const (&xr)[4], int L, int h, int G, int& row) {
    float4 v[4];
    load_rows4(xr, L, h, v);
    return group_dist_scatter4_v(yq, wq, v, L, h, G, row);
}

// The cnt <= 32 NE survivors as (distance key, draw index) sorted in registers (lane L holds
// sorted positions L NE .. L NE + NE - 1), then stored in order to the warp's sort buffer:
// no shared-memory traffic in the sort's stages.
template <int NE>
__device__ __forceinline__ void sort_keys_to_buffer(const float* kj, const int32_t* ij, int cnt,
                                                    unsigned long long* sbuf, int lane) {
    __syncwarp();
    unsigned long long v[NE];
#pragma unroll
    for (int i = 0; i < NE; ++i) {
        const int e = lane * NE + i;
        v[i] = e < cnt ? (((unsigned long long)f2key(kj[e]) << 32) | (uint32_t)ij[e]) : ~0ull;
    }
    warp_bitonic_sort_regs<NE>(v, lane);
#pragma unroll
    for (int i = 0; i < NE; ++i) sbuf[lane * NE + i] = v[i];
    __syncwarp();
}

__global__ void __launch_bounds__(256, 3) k_finalize(const __grid_constant__ BatchFin B) {
    extern __shared__ __align__(16) uint8_t fsm[];
    const int warps = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* hist = (uint32_t*)fsm + wid * 256;
    float* ys = (float*)(fsm + warps * 1024) + wid * 2 * MAXL;
    float* ws = ys + MAXL;
    unsigned long long* sbuf = (unsigned long long*)(fsm + warps * 1024 + warps * 2 * MAXL * 4) + (size_t)wid * B.sortcap;
    const int64_t g = (int64_t)blockIdx.x * warps + wid;
    if (g >= B.v_prefix[B.n_items]) return;
    int it = 0;
    while (it + 1 < B.n_items && g >= B.v_prefix[it + 1]) ++it;
    const FinItem& P = B.item[it];
    const int64_t gpos = g - B.v_prefix[it];               // voxel position
    if (P.rows && gpos >= (int64_t)*P.rcount) return;
    const int64_t j = P.rows ? (int64_t)P.rows[gpos] : gpos;   // packed row of the voxel
    if (j < 0) return;                                          // rescue padding
    const int64_t lr = P.rows ? gpos : j;                       // list row (the rescue lists by position)
    const int64_t vox = P.perm ? (int64_t)P.perm[j] : j;        // voxel of that row
    const int Cf = P.dyn_C ? *P.dyn_C : P.C;                    // list capacity
    const int C2f = P.dyn_C ? (P.C2 == P.C ? Cf : Cf / 2) : P.C2;
    float* kj = P.keys + lr * Cf;
    int32_t* ij = P.idx + lr * Cf;
    const int raw0 = P.cnt[lr], raw1 = P.cnt[lr + P.hstride];
    const int raw = raw0 | raw1;                          // an overflow flag from either half
    const int c0h = raw0 & 0x3FFFFFFF, c1h = raw1 & 0x3FFFFFFF;
    int cnt = c0h + c1h;
    // one contiguous list
    if (!(raw & 0x40000000)) merge_halves(kj, ij, C2f, c0h, c1h, lane);
    for (int l = lane; l < P.L; l += 32) {
        ys[l] = P.y[vox * P.ldy + l];
        ws[l] = P.w[l];
    }
    __syncwarp();
    int G = 1;
    while (4 * G < P.L) G <<= 1;
    const int R = 32 / G, grp = lane / G, h = lane % G;
    bool scan = (raw & 0x40000000) != 0;
    if (lane == 0) {                       // diagnostics: overflowed lists, short lists
        if (scan) atomicAdd(&B.status[4], 1);
        else if (cnt < P.k) atomicAdd(&B.status[5], 1);
        else if (cnt < P.kt) atomicAdd(&B.status[6], 1);
    }
    uint32_t K = 0;
    int n_less = -1, n_eq = -1;                   // keys below / at K (-1: not counted yet)
    // exact k-th distance of a net: bounds the true one (a rescued voxel starts from its first net's)
    float dbound = P.rows ? P.rq_dk[gpos] : __int_as_float(0x7F800000);
    if (!scan) {
        // 1. the net: every draw outside it has computed key > T_out (both halves dropped only
        // keys above their own thresholds)
        float T_out = fminf(P.thr[lr], P.thr[lr + P.hstride]);
        constexpr int NR = 4;
        float yq[4], wq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int l = 4 * h + q;
            yq[q] = l < P.L ? ys[l] : 0.0f;
            wq[q] = l < P.L ? ws[l] : 0.0f;
        }
        // split form: the net need not be the whole list.  The k smallest keys are re-scored
        // first (their rows gathered into sbuf); the largest of their exact distances, d1,
        // bounds the k-th distance from above, so every draw the certificate can ask for has
        // key <= need_key(d1).  The list is cut there and only the rest is re-scored.
        int n1 = 0;                          // entries of that first set, in sbuf: (distance, packed row)
        if (P.mode != ABC_FP32 && cnt > P.k) {
            const KthKey k1 = warp_select_exact(kj, cnt, P.k - 1, hist, (float*)sbuf, 2 * B.sortcap, lane);
            if (k1.n_less + k1.n_eq <= B.sortcap) {
                // the list read four rows of 32 at a time, their loads in flight together
                constexpr int RA = 4;
                for (int base = 0; base < cnt; base += 32 * RA) {
                    float kv[RA];
                    int32_t iv[RA];
#pragma unroll
                    for (int r = 0; r < RA; ++r) {
                        const int i = base + 32 * r + lane;
                        kv[r] = i < cnt ? kj[i] : __int_as_float(0x7F800000);
                        iv[r] = i < cnt ? ij[i] : 0;
                    }
#pragma unroll
                    for (int r = 0; r < RA; ++r) {
                        const int i = base + 32 * r + lane;
                        const bool in = i < cnt && f2key(kv[r]) <= k1.K;
                        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, in);
                        if (in) sbuf[n1 + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)iv[r];
                        n1 += __popc(bal);
                    }
                }
                __syncwarp();
                float d1 = 0.0f;
                // G >= 8: two groups of four rows per lane per iteration, all eight loads in
                // flight before either group's arithmetic (the same values as one group at a time)
                const int n1_pair = G >= 8 ? n1 - n1 % (2 * NR * R) : 0;
                for (int i0 = 0; i0 < n1_pair; i0 += 2 * NR * R) {
                    const float* xa[NR];
                    const float* xb[NR];
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        xa[r] = P.xs + (int64_t)(uint32_t)sbuf[i0 + r * R + grp] * P.ldxs;
                        xb[r] = P.xs + (int64_t)(uint32_t)sbuf[i0 + NR * R + r * R + grp] * P.ldxs;
                    }
                    float4 va[NR], vb[NR];
                    load_rows4(xa, P.L, h, va);
                    load_rows4(xb, P.L, h, vb);
                    int ra, rb;
                    const float da = group_dist_scatter4_v(yq, wq, va, P.L, h, G, ra);
                    const float db = group_dist_scatter4_v(yq, wq, vb, P.L, h, G, rb);
                    const int ia = i0 + ra * R + grp, ib = i0 + NR * R + rb * R + grp;
                    __syncwarp();
                    if ((h & ((G >> 2) - 1)) == 0) {
                        sbuf[ia] = ((unsigned long long)__float_as_uint(da) << 32) | (uint32_t)sbuf[ia];
                        sbuf[ib] = ((unsigned long long)__float_as_uint(db) << 32) | (uint32_t)sbuf[ib];
                        d1 = fmaxf(d1, fmaxf(da, db));
                    }
                    __syncwarp();
                }
                for (int i0 = n1_pair; i0 < n1; i0 += NR * R) {
                    const float* xr[NR];
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const int i = i0 + r * R + grp;
                        xr[r] = P.xs + (int64_t)(uint32_t)sbuf[i < n1 ? i : 0] * P.ldxs;
                    }
                    if (G >= 4) {
                        // the reduce-scatter form (the same value per row as the full butterfly)
                        int rr;
                        const float dv = group_dist_scatter4(yq, wq, xr, P.L, h, G, rr);
                        const int i = i0 + rr * R + grp;
                        __syncwarp();
                        if ((h & ((G >> 2) - 1)) == 0 && i < n1) {
                            sbuf[i] = ((unsigned long long)__float_as_uint(dv) << 32) | (uint32_t)sbuf[i];
                            d1 = fmaxf(d1, dv);
                        }
                    } else {
                        float d[NR];
                        group_dist_n<NR>(yq, wq, xr, P.L, h, G, d);
                        __syncwarp();
                        if (h == 0) {
#pragma unroll
                            for (int r = 0; r < NR; ++r) {
                                const int i = i0 + r * R + grp;
                                if (i < n1) {
                                    sbuf[i] = ((unsigned long long)__float_as_uint(d[r]) << 32) | (uint32_t)sbuf[i];
                                    d1 = fmaxf(d1, d[r]);
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d1 = fmaxf(d1, __shfl_xor_sync(0xFFFFFFFFu, d1, o));
                const float Tc = fminf(need_key(d1, P.ynorm[j], P.c0[j], P.dn[j],
                                                SplitCoef{P.cacc, 4.0f * (float)P.L * 0x1p-24f}), T_out);
                // keep K1 < key <= Tc (the first set is in sbuf), in place: a batch of four rows is
                // read before any of it is written, and writes stay below the next batch's reads
                int out = 0;
                for (int base = 0; base < cnt; base += 32 * RA) {
                    float kv[RA];
                    int32_t iv[RA];
#pragma unroll
                    for (int r = 0; r < RA; ++r) {
                        const int i = base + 32 * r + lane;
                        kv[r] = i < cnt ? kj[i] : __int_as_float(0x7F800000);
                        iv[r] = i < cnt ? ij[i] : 0;
                    }
                    __syncwarp();
#pragma unroll
                    for (int r = 0; r < RA; ++r) {
                        const int i = base + 32 * r + lane;
                        const bool keep = i < cnt && f2key(kv[r]) > k1.K && kv[r] <= Tc;
                        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
                        if (keep) {
                            const int pos = out + __popc(bal & ((1u << lane) - 1u));
                            kj[pos] = kv[r];
                            ij[pos] = iv[r];
                        }
                        out += __popc(bal);
                    }
                }
                __syncwarp();
                cnt = out;
                T_out = Tc;
            }
        }
        // 2. exact fp32 re-score of the (rest of the) net (list entries are packed draw rows, read
        // from the packed fp32 copy): G lanes per row, four rows per group in flight
        if (NR * R <= 32) {
            // row indices come a 32-row chunk at a time (lane t holds row cb + t), the next
            // chunk's already in flight, so a gather never waits on its own index load; the
            // chunk's global draw indices (ties break by them) are written back as it ends
            int cb = 0;
            int idx_cur = lane < cnt ? ij[lane] : 0;
            int idx_nxt = 32 + lane < cnt ? ij[32 + lane] : 0;
            int gx_cur = P.xperm ? P.xperm[idx_cur] : idx_cur;
            // G >= 8: two groups of four rows per lane per iteration (2 NR R <= 32 rows, inside
            // one 32-row index chunk), all eight loads in flight before either group's arithmetic
            const int cnt_pair = G >= 8 ? cnt - cnt % (2 * NR * R) : 0;
            int i0 = 0;
            for (; i0 < cnt_pair; i0 += 2 * NR * R) {
                if (i0 - cb >= 32) {
                    if (cb + lane < cnt) ij[cb + lane] = gx_cur;
                    cb += 32;
                    idx_cur = idx_nxt;
                    idx_nxt = cb + 32 + lane < cnt ? ij[cb + 32 + lane] : 0;
                    gx_cur = P.xperm ? P.xperm[idx_cur] : idx_cur;
                }
                const float* xa[NR];
                const float* xb[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int rowa = __shfl_sync(0xFFFFFFFFu, idx_cur, (i0 + r * R + grp - cb) & 31);
                    const int rowb = __shfl_sync(0xFFFFFFFFu, idx_cur, (i0 + NR * R + r * R + grp - cb) & 31);
                    xa[r] = P.xs + (int64_t)rowa * P.ldxs;
                    xb[r] = P.xs + (int64_t)rowb * P.ldxs;
                }
                float4 va[NR], vb[NR];
                load_rows4(xa, P.L, h, va);
                load_rows4(xb, P.L, h, vb);
                int ra, rb;
                const float da = group_dist_scatter4_v(yq, wq, va, P.L, h, G, ra);
                const float db = group_dist_scatter4_v(yq, wq, vb, P.L, h, G, rb);
                if ((h & ((G >> 2) - 1)) == 0) {
                    kj[i0 + ra * R + grp] = da;
                    kj[i0 + NR * R + rb * R + grp] = db;
                }
            }
            for (; i0 < cnt; i0 += NR * R) {
                if (i0 - cb >= 32) {
                    if (cb + lane < cnt) ij[cb + lane] = gx_cur;
                    cb += 32;
                    idx_cur = idx_nxt;
                    idx_nxt = cb + 32 + lane < cnt ? ij[cb + 32 + lane] : 0;
                    gx_cur = P.xperm ? P.xperm[idx_cur] : idx_cur;
                }
                const float* xr[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int row = __shfl_sync(0xFFFFFFFFu, idx_cur, (i0 + r * R + grp - cb) & 31);
                    xr[r] = P.xs + (int64_t)row * P.ldxs;
                }
                if (G >= 4) {
                    int rr;
                    const float dv = group_dist_scatter4(yq, wq, xr, P.L, h, G, rr);
                    const int i = i0 + rr * R + grp;
                    if ((h & ((G >> 2) - 1)) == 0 && i < cnt) kj[i] = dv;
                } else {
                    float d[NR];
                    group_dist_n<NR>(yq, wq, xr, P.L, h, G, d);
                    if (h == 0) {
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            const int i = i0 + r * R + grp;
                            if (i < cnt) kj[i] = d[r];
                        }
                    }
                }
            }
            if (cb + lane < cnt) ij[cb + lane] = gx_cur;
            __syncwarp();
        } else {
            for (int i0 = 0; i0 < cnt; i0 += NR * R) {
                const float* xr[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int i = i0 + r * R + grp;
                    xr[r] = P.xs + (int64_t)ij[i < cnt ? i : cnt - 1] * P.ldxs;
                }
                float d[NR];
                group_dist_n<NR>(yq, wq, xr, P.L, h, G, d);
                __syncwarp();
                if (h == 0) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const int i = i0 + r * R + grp;
                        if (i < cnt) kj[i] = d[r];
                    }
                }
            }
            __syncwarp();
            // back to global draw indices (ties break by them)
            if (P.xperm) {
                for (int i = lane; i < cnt; i += 32) ij[i] = P.xperm[ij[i]];
                __syncwarp();
            }
        }
        // the first set joins the re-scored net: exact distances and global draw indices
        if (n1 > 0) {
            for (int i = lane; i < n1; i += 32) {
                const unsigned long long e = sbuf[i];
                const int32_t row = (int32_t)(uint32_t)e;
                kj[cnt + i] = __uint_as_float((uint32_t)(e >> 32));
                ij[cnt + i] = P.xperm ? P.xperm[row] : row;
            }
            cnt += n1;
            __syncwarp();
        }
        // 3. exact k-th distance and the certificate
        bool cert = false;
        if (cnt >= P.k) {
            const KthKey kth = warp_select_exact(kj, cnt, P.k - 1, hist, (float*)sbuf, 2 * B.sortcap, lane);
            K = kth.K;
            n_less = kth.n_less;
            n_eq = kth.n_eq;
            const float dk = key2f(K);
            dbound = fminf(dbound, dk);
            const float yn = P.ynorm[j];
            float need;
            const float slack = 4.0f * (float)P.L * 0x1p-24f;
            if (P.mode == ABC_FP32) {
                const float ry = sqrtf(yn);
                const float R = ry + sqrtf(dk * (1.0f + slack)) + 1e-30f;
                need = dk * (1.0f + slack) - yn * (1.0f - slack) + err_bound(3.0f * 0x1p-16f + P.cacc, ry, R);
            } else {
                // every draw at exact distance <= d_k has key <= need_key(d_k)
                need = need_key(dk, yn, P.c0[j], P.dn[j], SplitCoef{P.cacc, slack});
            }
            cert = (T_out >= 2.9e38f || T_out >= need) && !((B.force_rescue & 1) && P.rq_rows) &&
                   !((B.force_rescue & 2) && P.rows);
        }
        if (!cert) {
            // split form, first pass: the net's d_k bounds the exact k-th distance, so
            // need_key(d_k) is a threshold that collects every draw the certificate can ask
            // for; the voxel is queued for a second tensor-core pass with it, whose own
            // finalize writes its outputs.  Otherwise (queue full, or the second pass) the
            // exact scan below resolves it.
            if (P.rq_rows && cnt >= P.k) {
                int pos = 0;
                if (lane == 0) pos = atomicAdd(P.rq_count, 1);
                pos = __shfl_sync(0xFFFFFFFFu, pos, 0);
                if (pos < P.rq_cap) {
                    if (lane == 0) {
                        P.rq_rows[pos] = (int32_t)j;
                        P.rq_dk[pos] = dbound;
                        P.rq_thr[pos] = need_key(dbound, P.ynorm[j], P.c0[j], P.dn[j],
                                                 SplitCoef{P.cacc, 4.0f * (float)P.L * 0x1p-24f});
                        atomicAdd(&B.status[3], 1);
                    }
                    return;
                }
            }
            scan = true;
        }
    }
    if (scan) {
        // exact fp32 scan (candidate list rebuilt with exact keys) of every draw that can
        // be within the net's exact k-th distance: with ordered draws, only the 64-draw
        // tiles whose segment-feature bound does not exceed it
        if (lane == 0) atomicAdd(&B.status[1], 1);
        cnt = 0;
        float thr = dbound;
        auto take_row = [&](int64_t n, const float* xrow, int32_t gidx) {
            const float d = n < P.N ? lane_dist(ys, ws, xrow, P.L, G) : __int_as_float(0x7F800000);
            const bool take = n < P.N && d <= thr;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, take);
            if (take) {
                const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                kj[pos] = d;
                ij[pos] = gidx;
            }
            cnt += __popc(bal);
            if (cnt > Cf - 32) {
                __syncwarp();
                const uint32_t T = warp_select(kj, cnt, P.k - 1, 4, hist, lane);
                const int q = warp_compact(kj, ij, cnt, T, Cf - 64, lane);
                cnt = q < Cf - 64 ? q : Cf - 64;
                thr = key2f(T);
            }
        };
        if (P.tbox) {
            const float db = dbound < 3.0e38f ? dbound * (1.0f + 0x1p-10f) : 3.0e38f;
            const float f0 = P.fy[3 * j], f1 = P.fy[3 * j + 1], f2 = P.fy[3 * j + 2];
            for (int64_t t0 = 0; t0 < P.nt64; t0 += 32) {
                const int64_t t = t0 + lane;
                bool keep = false;
                if (t < P.nt64 && t * 64 < P.N) {
                    float lb = 0.0f;
                    const float fv[3] = {f0, f1, f2};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float xl = P.tbox[6 * t + 2 * c], xh = P.tbox[6 * t + 2 * c + 1];
                        const float slack = 0x1p-18f * (fabsf(xl) + fabsf(xh) + 2.0f * fabsf(fv[c]));
                        const float gap = fmaxf(fmaxf(xl - fv[c], fv[c] - xh) - slack, 0.0f);
                        if (P.Wc[c] > 0.0f) lb += gap * gap / P.Wc[c];
                    }
                    keep = lb * (1.0f - 0x1p-10f) <= db;
                }
                uint32_t km = __ballot_sync(0xFFFFFFFFu, keep);
                while (km) {
                    const int b = __ffs(km) - 1;
                    km &= km - 1;
#pragma unroll 1
                    for (int hh = 0; hh < 2; ++hh) {
                        const int64_t n = (t0 + b) * 64 + hh * 32 + lane;      // packed draw row
                        const int64_t nn = n < P.N ? n : 0;
                        take_row(n, P.xs + nn * P.ldxs, P.xperm ? P.xperm[nn] : (int32_t)nn);
                    }
                }
            }
        } else {
            for (int64_t base = 0; base < P.N; base += 32) {
                const int64_t n = base + lane;
                take_row(n, P.x + (n < P.N ? n : 0) * P.ldx, (int32_t)n);
            }
        }
        __syncwarp();
        K = cnt >= P.k ? warp_select(kj, cnt, P.k - 1, 4, hist, lane) : 0xFFFFFFFFu;
    }
    // 4. keep everything at or below the exact k-th distance, sort by (distance, index)
    if (cnt > P.k) {
        if (n_less < 0) {
            const KthKey c = warp_count_key(kj, cnt, K, lane);
            n_less = c.n_less;
            n_eq = c.n_eq;
        }
        if (n_less + n_eq > P.sortcap) {
            // more entries at the k-th distance than the sort holds: keep the ties with the
            // lowest draw indices (global by now), chosen by a selection on the indices
            if (lane == 0) atomicAdd(&B.status[2], 1);
            const uint32_t Ti = warp_select_tie_index(kj, ij, cnt, K, P.k - n_less - 1, hist, lane);
            cnt = warp_compact_ties(kj, ij, cnt, K, Ti, lane);
        } else {
            const int gq = warp_compact(kj, ij, cnt, K, P.sortcap, lane);
            cnt = gq < P.sortcap ? gq : P.sortcap;
        }
    }
    int n2 = 32;
    while (n2 < cnt) n2 <<= 1;
    // 256 survivors (k up to 248) sort in registers; 512 in registers spilled and measured
    // slower on the brain volume (k = 500), so larger sorts stay in shared memory
    if (n2 == 256) {
        sort_keys_to_buffer<8>(kj, ij, cnt, sbuf, lane);
    } else {
        for (int i = lane; i < n2; i += 32)
            sbuf[i] = i < cnt ? (((unsigned long long)f2key(kj[i]) << 32) | (uint32_t)ij[i]) : ~0ull;
        warp_bitonic_sort(sbuf, n2, lane);
    }
    for (int r = lane; r < P.k; r += 32) {
        const unsigned long long e = r < cnt ? sbuf[r] : ~0ull;
        P.out_idx[vox * P.k + r] = r < cnt ? (int32_t)(uint32_t)e : -1;
        P.out_dist[vox * P.k + r] = r < cnt ? key2f((uint32_t)(e >> 32)) : __int_as_float(0x7F800000);
    }
}

// Kernel parameter blocks must fit the 32 KB parameter space.
static_assert(sizeof(BatchTc) <= 32000, "BatchTc exceeds the kernel parameter space");
static_assert(sizeof(BatchFin) <= 32000, "BatchFin exceeds the kernel parameter space");
static_assert(sizeof(BatchPilot) <= 32000, "BatchPilot exceeds the kernel parameter space");

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
// Test hook (abc_debug_inject_stall): bound on the fused kernel's barrier waits and
// the draw-tile sequence number its TMA producers withhold (-1: none).
uint64_t g_wait_ns = WAIT_NS_DEFAULT;
int64_t g_withhold = -1;
int g_force_rescue = 0;        // test hook bits (abc_debug_force_rescue)
int g_order_mode = 0;          // row order: 0 by scan size, 1 Morton, 2 k-d (abc_debug_order)
cudaEvent_t g_prof_start = nullptr, g_prof_stop = nullptr;
int g_last_resident = 0;     // residency of the last configured fused-kernel variant
int64_t g_last_grid = 0;     // grid of the last fused-kernel launch

// Records a timing event on s; inside a stream capture it becomes a record node
// of the graph (an ordinary record there would only express a dependency).
cudaError_t record_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t r = cudaStreamIsCapturing(s, &cs);
    if (r != cudaSuccess) return r;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                               : cudaEventRecord(e, s);
}

int get_encoder() {
    if (g_encode) return ABC_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    VPET_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (!fn || q != cudaDriverEntryPointSuccess) {
        vpet::set_error("cuTensorMapEncodeTiled not available from the driver");
        return ABC_ERR_CUDA;
    }
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return ABC_OK;
}

// Rows of Kp bf16 (128-byte swizzle), box {64, box_rows}; row_step > 1 gives a
// view of every row_step-th row (pilot passes).
int make_tmap(CUtensorMap* m, void* base, int64_t rows, int Kp, int box_rows, int64_t row_step) {
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2 * (cuuint64_t)row_step};
    const cuuint32_t box[2] = {(cuuint32_t)KBLK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        vpet::set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return ABC_ERR_CUDA;
    }
    return ABC_OK;
}

// TMA ring depth per shape: as deep as shared memory allows next to the A tile, the key rows
// (if any) and the epilogue warps' histograms; two K-blocks of 128-draw tiles without rows:
// two stages, so that two CTAs fit on an SM
constexpr int stages_for(int nkb, int bn, bool topr) {
    return nkb == 1 ? (bn == 128 ? 3 : 4)
                    : (nkb == 2 ? (topr ? (bn == 128 ? 4 : 3) : (bn == 128 ? 2 : 4)) : (bn == 128 ? 2 : 4));
}

size_t tc_smem_bytes(int nkb, int bn, bool topr) {
    const int S = stages_for(nkb, bn, topr);
    const int epi = tc_epi_warps(topr, bn);
    return 1024 + (size_t)nkb * A_KBLK_BYTES + (size_t)S * nkb * bn * KBLK * 2 +
           (tc_rows(nkb, topr) ? (size_t)32 * epi * ROW_LD * 4 : 0) +
           (size_t)epi * 256 * 4 + (2 * S + 14) * 8;
}

int num_sms() {
    static int sms[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!sms[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        sms[dev] = v;
    }
    return sms[dev];
}

template <int NKB, int BN, bool DUMP, bool TOPR>
int launch_tc(const BatchTc& P, int ctas_per_sm, cudaStream_t s) {
    constexpr int S = stages_for(NKB, BN, TOPR);
    const size_t smem = tc_smem_bytes(NKB, BN, TOPR);
    // kernel attributes are per device: configured once for each device that launches
    static bool configured_dev[64] = {};
    static int max_resident_dev[64] = {};
    int cur = 0;
    VPET_CUDA(cudaGetDevice(&cur));
    VPET_ARG(cur >= 0 && cur < 64, "device ordinal %d out of range", cur);
    bool& configured = configured_dev[cur];
    int& max_resident = max_resident_dev[cur];
    if (!configured) {
        VPET_CUDA(cudaFuncSetAttribute(k_tc_topk<NKB, S, BN, DUMP, TOPR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        // all of the unified L1 / shared storage as shared memory, so that the
        // residency the tuning asks for is actually available
        VPET_CUDA(cudaFuncSetAttribute(k_tc_topk<NKB, S, BN, DUMP, TOPR>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared));
        // residency from the limits that apply: shared memory, registers, TMEM columns
        cudaFuncAttributes fa;
        VPET_CUDA(cudaFuncGetAttributes(&fa, k_tc_topk<NKB, S, BN, DUMP, TOPR>));
        int dev = 0, smem_sm = 0, resv = 0;
        VPET_CUDA(cudaGetDevice(&dev));
        VPET_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        VPET_CUDA(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
        const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + resv);
        const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
        const int by_regs = 65536 / (regs_warp * (tc_threads(TOPR, BN) / 32));
        const int by_tmem = 512 / (2 * BN);
        max_resident = by_smem < by_regs ? by_smem : by_regs;
        if (max_resident > by_tmem) max_resident = by_tmem;
        if (max_resident < 1) max_resident = 1;
        g_last_resident = max_resident;
        configured = true;
    }
    const int per_sm = ctas_per_sm < max_resident ? ctas_per_sm : max_resident;
    const int64_t total = P.vt_prefix[P.n_items];
    int64_t grid = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    if (grid > total) grid = total;
    if (grid < 1) return ABC_OK;
    g_last_grid = grid;
    k_tc_topk<NKB, S, BN, DUMP, TOPR><<<(unsigned)grid, tc_threads(TOPR, BN), smem, s>>>(P);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

// topr: every item of the batch is a top-r pilot (rsel > 0)
template <bool DUMP>
int dispatch_tc(int nkb, int bn, const BatchTc& P, int ctas_per_sm, cudaStream_t s, bool topr = false) {
    if (bn == 128) {
        switch (nkb) {
            case 1: return topr ? launch_tc<1, 128, false, true>(P, ctas_per_sm, s) : launch_tc<1, 128, DUMP, false>(P, ctas_per_sm, s);
            case 2: return topr ? launch_tc<2, 128, false, true>(P, ctas_per_sm, s) : launch_tc<2, 128, DUMP, false>(P, ctas_per_sm, s);
            case 3: return topr ? launch_tc<3, 128, false, true>(P, ctas_per_sm, s) : launch_tc<3, 128, DUMP, false>(P, ctas_per_sm, s);
        }
    } else if (!DUMP && bn == 64) {
        switch (nkb) {
            case 1: return topr ? launch_tc<1, 64, false, true>(P, ctas_per_sm, s) : launch_tc<1, 64, false, false>(P, ctas_per_sm, s);
            case 2: return topr ? launch_tc<2, 64, false, true>(P, ctas_per_sm, s) : launch_tc<2, 64, false, false>(P, ctas_per_sm, s);
            case 3: return topr ? launch_tc<3, 64, false, true>(P, ctas_per_sm, s) : launch_tc<3, 64, false, false>(P, ctas_per_sm, s);
        }
    }
    vpet::set_error("unsupported tile shape (K-blocks %d, BN %d)", nkb, bn);
    return ABC_ERR_UNSUPPORTED;
}

float error_coef(const Layout& lay) {
    // ABC_FP32: |d' error| <= cE (2 ||yh|| R + R^2) for a draw with ||xh|| <= R.  bf16
    // hi + lo of each operand leaves |a - a_hi - a_lo| <= 2^-16 |a|, |a_lo| <= 2^-8 |a|, so the
    // three products miss at most 3 * 2^-16 |a b|; plus fp32 accumulation over Kp terms, the
    // fp32 norm and the fp32 centring / scaling of the operands.
    return 3.0f * 0x1p-16f + (float)(3 * lay.Kp + lay.L + 16) * 0x1p-24f;
}

// Split form: the coefficients of need_key / dist_ub.
SplitCoef split_coef(const Layout& lay) {
    return SplitCoef{(float)(3 * lay.Kp + lay.L + 16) * 0x1p-24f, 4.0f * (float)lay.L * 0x1p-24f};
}

// One scan of a batch as the host sees it.
struct ScanSpec {
    const float* y;
    int64_t J;
    int ldy;
    const float* x;
    int64_t N;
    int ldx;
    int L;
    const float* w;
    int k;
    int32_t* idx;
    float* dist;
};

int validate(const ScanSpec& c, int mode) {
    VPET_ARG(c.J >= 1 && c.N >= 1, "discrepancy/top-k: J and N must be >= 1");
    VPET_ARG(c.N < ((int64_t)1 << 31), "discrepancy/top-k: N must be < 2^31");
    VPET_ARG(c.L >= 1 && c.L <= 61, "discrepancy/top-k: L must be in 1..61 (got %d)", c.L);
    VPET_ARG(c.k >= 1 && c.k <= 2048 && c.k <= c.N, "discrepancy/top-k: need 1 <= k <= min(N, 2048)");
    VPET_ARG(mode == ABC_FP32 || mode == ABC_BF16_RESCORE || mode == ABC_SPLIT_DRAWS,
             "discrepancy/top-k: unknown precision %d", mode);
    VPET_ARG(c.y && c.x && c.w, "discrepancy/top-k: null pointer");
    VPET_ARG(c.ldy >= c.L && c.ldx >= c.L && c.ldx % 4 == 0 && c.ldy % 4 == 0,
             "discrepancy/top-k: ldy, ldx must be >= L and multiples of 4");
    VPET_ARG(((uintptr_t)c.y & 15) == 0 && ((uintptr_t)c.x & 15) == 0, "discrepancy/top-k: y, x must be 16-byte aligned");
    bool any = false;
    for (int l = 0; l < c.L; ++l) {
        VPET_ARG(c.w[l] >= 0.0f && c.w[l] == c.w[l], "discrepancy/top-k: weights must be >= 0");
        any |= c.w[l] > 0.0f;
    }
    VPET_ARG(any, "discrepancy/top-k: all weights are zero");
    return ABC_OK;
}

int check_tuning(const Tuning& t) {
    VPET_ARG(t.bn == 64 || t.bn == 128, "tuning: bn must be 64 or 128");
    VPET_ARG(t.ctas_per_sm >= 1 && t.ctas_per_sm <= 4, "tuning: ctas_per_sm must be in 1..4");
    VPET_ARG(t.pilot_stride == 8 || t.pilot_stride == 16 || t.pilot_stride == 32, "tuning: pilot_stride must be 8, 16 or 32");
    VPET_ARG(t.pilot_factor >= 1.25f && t.pilot_factor <= 4.0f, "tuning: pilot_factor must be in [1.25, 4]");
    return ABC_OK;
}

// Workspace of a batch: a 256-byte status block, then one section per scan.
struct BatchLayout {
    int n;
    Layout lay[MAX_ITEMS];
    size_t off[MAX_ITEMS];
    size_t total;
};

// Split-form memory choices per scan, each within a budget:
//  - candidate-list capacity 12 m k entries, m in {1, 2, 4}: a single scan takes the largest m
//    whose lists fit LIST_BYTES_SINGLE; in a batch the smallest scans are raised first while
//    the extra list bytes fit LIST_EXTRA_BYTES_BATCH (a small scan's lists are cheap, and its
//    voxels are the most varied, so its nets are the longest);
//  - centring groups: up to MAX_GROUPS per scan, each at least GROUP_MIN_TILES voxel tiles;
//    every group costs a copy of the draw operand, so groups are added one at a time to the
//    scan with the most voxels per copy byte, discounted by the groups it has (gain
//    J / (G (G + 1)) per byte), while all copies fit the budget.  Each copy also costs the
//    main pass L2 reuse (CTAs working on different groups read different copies): for one
//    scan about 2 GB of copies (the brain volume: 4 of 512 MB) measured best, a batch of many
//    small, varied scans needs far more (the 64-scan batch: 64 GB).
constexpr double LIST_BYTES_SINGLE = 32.0e9, LIST_EXTRA_BYTES_BATCH = 16.0e9;
constexpr double GROUP_COPIES_BYTES_SINGLE = 2.1e9, GROUP_COPIES_BYTES_BATCH = 64.0e9;
constexpr int64_t GROUP_MIN_TILES = 2;

void make_batch_layout(const ScanSpec* sc, int n, int mode, const Tuning& tu, BatchLayout* B, bool grouped = true) {
    B->n = n;
    int kp = 0;
    for (int i = 0; i < n; ++i) {
        const int w = make_layout(sc[i].J, sc[i].N, sc[i].L, sc[i].k, mode, tu).Kp;
        if (w > kp) kp = w;
    }
    const bool split = mode != ABC_FP32;
    auto list_bytes = [&](int i, int m) { return (double)sc[i].J * (12.0 * m * sc[i].k + 256.0) * 8.0; };
    int mult[MAX_ITEMS];
    for (int i = 0; i < n; ++i) mult[i] = 1;
    if (split && n == 1) {
        for (int m = 4; m > 1; m /= 2)
            if (list_bytes(0, m) <= LIST_BYTES_SINGLE) {
                mult[0] = m;
                break;
            }
    } else if (split) {
        int by_size[MAX_ITEMS];
        for (int i = 0; i < n; ++i) by_size[i] = i;
        for (int a = 1; a < n; ++a)
            for (int b = a; b > 0 && sc[by_size[b]].J < sc[by_size[b - 1]].J; --b) {
                const int t = by_size[b];
                by_size[b] = by_size[b - 1];
                by_size[b - 1] = t;
            }
        double extra = 0.0;
        for (int a = 0; a < n; ++a) {
            const int i = by_size[a];
            for (int m = 4; m > 1; m /= 2) {
                const double e = list_bytes(i, m) - list_bytes(i, 1);
                if (extra + e <= LIST_EXTRA_BYTES_BATCH) {
                    mult[i] = m;
                    extra += e;
                    break;
                }
            }
        }
    }
    int groups[MAX_ITEMS], gmax[MAX_ITEMS];
    double copy_bytes[MAX_ITEMS], total = 0.0;
    for (int i = 0; i < n; ++i) {
        const int64_t g = vpet_ceil_div(sc[i].J > 0 ? sc[i].J : 1, GROUP_MIN_TILES * BM);
        gmax[i] = (!split || !grouped) ? 1 : (int)(g < MAX_GROUPS ? g : MAX_GROUPS);
        groups[i] = 1;
        copy_bytes[i] = (double)vpet_round_up(sc[i].N > 0 ? sc[i].N : 1, 128) * kp * 2.0;
        total += copy_bytes[i];
    }
    const double budget = n == 1 ? GROUP_COPIES_BYTES_SINGLE : GROUP_COPIES_BYTES_BATCH;
    for (;;) {
        int best = -1;
        double best_gain = 0.0;
        for (int i = 0; i < n; ++i) {
            if (groups[i] >= gmax[i] || total + copy_bytes[i] > budget) continue;
            const double gain = (double)sc[i].J / ((double)groups[i] * (groups[i] + 1)) / copy_bytes[i];
            if (gain > best_gain) {
                best_gain = gain;
                best = i;
            }
        }
        if (best < 0) break;
        groups[best] += 1;
        total += copy_bytes[best];
    }
    // one K-width per launch: every scan is laid out at the widest
    size_t o = 256;
    for (int i = 0; i < n; ++i) {
        B->lay[i] = make_layout(sc[i].J, sc[i].N, sc[i].L, sc[i].k, mode, tu, kp, mult[i], groups[i]);
        B->off[i] = o;
        o = align256(o + B->lay[i].total);
    }
    B->total = o;
}

// Every section of a scan's layout lies after the previous one and inside the scan's total.
bool layout_consistent(const Layout& L) {
    const size_t off[] = {L.off_mu, L.off_part, L.off_ynorm, L.off_c0, L.off_dn, L.off_a, L.off_b, L.off_keys,
                          L.off_idx, L.off_cnt, L.off_thr, L.off_thr0, L.off_perm, L.off_feat, L.off_hist,
                          L.off_xperm, L.off_xfeat, L.off_xhist, L.off_fy, L.off_fx, L.off_tbox, L.off_ktile,
                          L.off_kcount, L.off_xs, L.off_w, L.off_tgroup, L.off_rq, L.off_rrow, L.off_rthr,
                          L.off_rq2, L.off_rtg, L.off_rcnt, L.off_rthrh, L.off_ra};
    const size_t len[] = {(size_t)L.G * MAXL * 4, (size_t)L.G * L.npart * MAXL * 4, (size_t)L.Jp * 4, (size_t)L.Jp * 4,
                          (size_t)L.Jp * 4, (size_t)L.Jp * L.Kp * 2, (size_t)L.G * L.Np * L.Kp * 2,
                          (size_t)L.lrows * L.C * 4, (size_t)L.lrows * L.C * 4, (size_t)2 * L.Jp * 4, (size_t)2 * L.Jp * 4, (size_t)L.Jp * 4,
                          (size_t)L.Jp * 4, (size_t)3 * L.Jp * 4 + 32, (size_t)(ORDER_BUCKETS + ORDER_BUCKETS / 1024) * 4,
                          (size_t)L.Np * 4, (size_t)3 * L.Np * 4 + 32, (size_t)(ORDER_BUCKETS + ORDER_BUCKETS / 1024) * 4,
                          (size_t)3 * L.Jp * 4, (size_t)3 * L.Np * 4, (size_t)6 * L.nt64 * 4,
                          (size_t)L.nvt * L.nt64 * 4, (size_t)L.nvt * 4, (size_t)L.Np * L.ldxs * 4, MAXL * 4,
                          (size_t)L.nvt * 4, (size_t)(2 + 3 * L.G + 2) * 4, (size_t)L.rcapa * 4, (size_t)L.rcapa * 8,
                          (size_t)L.rcapa * 12, (size_t)(L.rcapa / BM + 1) * 4, (size_t)L.rcapa * 8,
                          (size_t)L.rcapa * 8, (size_t)L.rcapa * L.Kp * 2};
    const int n = (int)(sizeof off / sizeof off[0]);
    for (int i = 0; i < n; ++i) {
        if (off[i] + len[i] > (i + 1 < n ? off[i + 1] : L.total)) return false;
        if (i > 0 && off[i] < off[i - 1]) return false;
    }
    // the rescue pass's lists (rcapa rows of Cr) lie in the candidate-list space
    if (L.rcapa > 0 && (L.Cr < L.C || L.Cr % 2 || (double)L.Cr * L.rcapa > (double)L.lrows * L.C)) return false;
    return true;
}

// Voxels the first finalize may queue for the rescue pass, the same for every kernel that
// reads the queue (the test hook's bit 4 limits it to a quarter of the voxels).
int64_t queue_cap(const Layout& L) { return (g_force_rescue & 4) && L.rcap > L.J / 4 ? L.J / 4 : L.rcap; }

int run_batch(const ScanSpec* sc, int n, int mode, const Tuning& tu_in, void* ws, size_t ws_bytes, float* dump,
              int64_t ld_dump, cudaStream_t s) {
    VPET_ARG(n >= 1 && n <= MAX_ITEMS, "batch: 1..%d scans per call (got %d)", MAX_ITEMS, n);
    Tuning tu = tu_in;
    if (dump) tu.bn = 128;       // the key dump is only instantiated for 128-draw tiles
    int rc = check_tuning(tu);
    if (rc) return rc;
    for (int i = 0; i < n; ++i)
        if ((rc = validate(sc[i], mode))) return rc;
    BatchLayout BL;
    make_batch_layout(sc, n, mode, tu, &BL, dump == nullptr);   // the key dump keeps one centre
    for (int i = 0; i < n; ++i)
        if (!layout_consistent(BL.lay[i])) {
            vpet::set_error("discrepancy/top-k: internal workspace layout error (scan %d)", i);
            return ABC_ERR_WORKSPACE;
        }
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < BL.total) {
        vpet::set_error("discrepancy/top-k: workspace needs %zu bytes, 256-aligned (got %zu)", BL.total, ws_bytes);
        return ABC_ERR_WORKSPACE;
    }
    if (!dump)
        for (int i = 0; i < n; ++i) VPET_ARG(sc[i].idx && sc[i].dist, "discrepancy/top-k: null output");
    if ((rc = get_encoder())) return rc;
    uint8_t* wsb = (uint8_t*)ws;
    int32_t* status = (int32_t*)wsb;
    unsigned long long* counters = (unsigned long long*)(wsb + 64);   // one work counter per fused launch
    VPET_CUDA(cudaMemsetAsync(status, 0, 256, s));
    const int nkb = BL.lay[0].nkb;

    // per scan: centring, packing, tensor maps
    BatchTc T;                 // kernel parameter blocks (copied into each launch)
    BatchPilot PB;
    BatchFin F;
    struct Ptrs {
        float *mu, *part, *ynorm, *c0, *dn, *keys, *thr, *thr0, *feat, *xfeat, *fy, *fx, *tbox;
        int32_t *perm, *xperm, *ktile, *kcount;
        float* xs;
        uint32_t *mm, *hist, *xmm, *xhist;
        __nv_bfloat16 *A, *B, *RA;
        int32_t *idx, *cnt;
        float* wdev;
        int32_t *rq, *rrow, *tgroup, *rrow2, *rtg, *rcnt;
        float *rthr, *rthr2, *rdk2, *rthrh;
    } ptr[MAX_ITEMS];
    for (int i = 0; i < n; ++i) {
        const Layout& L = BL.lay[i];
        uint8_t* base = wsb + BL.off[i];
        Ptrs& p = ptr[i];
        p.mu = (float*)(base + L.off_mu);
        p.part = (float*)(base + L.off_part);
        p.ynorm = (float*)(base + L.off_ynorm);
        p.c0 = (float*)(base + L.off_c0);
        p.dn = (float*)(base + L.off_dn);
        p.A = (__nv_bfloat16*)(base + L.off_a);
        p.B = (__nv_bfloat16*)(base + L.off_b);
        p.keys = (float*)(base + L.off_keys);
        p.idx = (int32_t*)(base + L.off_idx);
        p.cnt = (int32_t*)(base + L.off_cnt);
        p.thr = (float*)(base + L.off_thr);
        p.thr0 = (float*)(base + L.off_thr0);
        p.perm = (int32_t*)(base + L.off_perm);
        p.feat = (float*)(base + L.off_feat);
        p.mm = (uint32_t*)(p.feat + 3 * L.Jp);
        p.hist = (uint32_t*)(base + L.off_hist);
        p.xperm = (int32_t*)(base + L.off_xperm);
        p.xfeat = (float*)(base + L.off_xfeat);
        p.xmm = (uint32_t*)(p.xfeat + 3 * L.Np);
        p.xhist = (uint32_t*)(base + L.off_xhist);
        p.fy = (float*)(base + L.off_fy);
        p.fx = (float*)(base + L.off_fx);
        p.tbox = (float*)(base + L.off_tbox);
        p.ktile = (int32_t*)(base + L.off_ktile);
        p.kcount = (int32_t*)(base + L.off_kcount);
        p.xs = (float*)(base + L.off_xs);
        p.wdev = (float*)(base + L.off_w);
        p.rq = (int32_t*)(base + L.off_rq);
        p.rrow = (int32_t*)(base + L.off_rrow);
        p.rthr = (float*)(base + L.off_rthr);
        p.RA = (__nv_bfloat16*)(base + L.off_ra);
        p.tgroup = (int32_t*)(base + L.off_tgroup);
        p.rrow2 = (int32_t*)(base + L.off_rq2);
        p.rthr2 = (float*)(p.rrow2 + L.rcapa);
        p.rdk2 = p.rthr2 + L.rcapa;
        p.rtg = (int32_t*)(base + L.off_rtg);
        p.rcnt = (int32_t*)(base + L.off_rcnt);
        p.rthrh = (float*)(base + L.off_rthrh);
        Weights W;
        memset(&W, 0, sizeof W);
        for (int l = 0; l < L.L; ++l) {
            W.w[l] = sc[i].w[l];
            W.sw[l] = sqrtf(sc[i].w[l]);
        }
        VPET_CUDA(cudaMemsetAsync(p.cnt, 0, (size_t)2 * L.Jp * sizeof(int32_t), s));
        VPET_CUDA(cudaMemsetAsync(p.rq, 0, (size_t)(2 + 3 * L.G + 2) * sizeof(int32_t), s));
        if (L.rcapa > 0) VPET_CUDA(cudaMemsetAsync(p.rcnt, 0, (size_t)2 * L.rcapa * sizeof(int32_t), s));
        const bool order = dump == nullptr && L.J > 1;   // the debug dump keeps voxel order
        // a large scan orders voxels and draws by k-d splits (tighter tile boxes, fewer tiles in
        // every pass), a small one by the Morton key (fewer launches)
        const bool kd = g_order_mode == 2 || (g_order_mode == 0 && (double)L.J * (double)L.N >= KD_MIN_PAIRS);
        bool kd_done = false;
        if (order && kd &&
            (rc = kd_order(sc[i].y, L.J, sc[i].ldy, L.L, W, 0, 1, p.A, (size_t)L.Jp * L.Kp * 2, p.perm, status, s,
                           kd_done)))
            return rc;
        if (order && !kd_done) {
            k_order_init<<<(unsigned)vpet_ceil_div(ORDER_BUCKETS, 256), 256, 0, s>>>(p.mm, p.hist);
            VPET_LAUNCH_CHECK();
            const unsigned gb = (unsigned)vpet_ceil_div(L.J, 256);
            k_order_features<<<gb, 256, 0, s>>>(sc[i].y, L.J, sc[i].ldy, L.L, W, p.feat, p.mm);
            VPET_LAUNCH_CHECK();
            k_order_hist<<<gb, 256, 0, s>>>(p.feat, p.mm, L.J, 0, 1, p.hist);
            VPET_LAUNCH_CHECK();
            k_order_scan_sums<<<SCAN_BLOCKS, 1024, 0, s>>>(p.hist, p.hist + ORDER_BUCKETS);
            k_order_scan_top<<<1, 1024, 0, s>>>(p.hist + ORDER_BUCKETS);
            k_order_scan<<<SCAN_BLOCKS, 1024, 0, s>>>(p.hist, p.hist + ORDER_BUCKETS);
            VPET_LAUNCH_CHECK();
            k_order_scatter<<<gb, 256, 0, s>>>(p.feat, p.mm, L.J, 0, 1, p.hist, p.perm);
            VPET_LAUNCH_CHECK();
        }
        // the centring groups' means (runs of the packed voxel order), and each voxel tile's group
        k_colmean_part<<<(unsigned)(L.G * L.npart), 256, 0, s>>>(sc[i].y, L.J, sc[i].ldy, L.L, p.part, L.npart,
                                                                 order ? p.perm : nullptr, L.Jg);
        VPET_LAUNCH_CHECK();
        k_colmean_final<<<(unsigned)L.G, MAXL, 0, s>>>(p.part, L.npart, L.J, L.Jg, p.mu, W, p.wdev);
        VPET_LAUNCH_CHECK();
        k_tile_groups<<<(unsigned)vpet_ceil_div(L.nvt, 256), 256, 0, s>>>(p.tgroup, L.nvt, L.Jg);
        VPET_LAUNCH_CHECK();
        k_pack_y<<<(unsigned)vpet_ceil_div(L.Jp, 8), 256, 0, s>>>(sc[i].y, L.J, L.Jp, sc[i].ldy, L.L, L.Kp, mode, W,
                                                                  p.mu, L.Jg, order ? p.perm : nullptr, p.A, p.ynorm,
                                                                  p.c0, p.dn, p.fy);
        VPET_LAUNCH_CHECK();
        // draws in the same kind of order (alike draws in the same tiles, so that tile boxes are tight)
        const bool xorder = dump == nullptr && L.N > 1;
        bool xkd_done = false;
        if (xorder && kd &&
            (rc = kd_order(sc[i].x, L.N, sc[i].ldx, L.L, W, L.nlev, tu.pilot_stride, p.B,
                           (size_t)L.G * L.Np * L.Kp * 2, p.xperm, status, s, xkd_done)))
            return rc;
        if (xorder && !xkd_done) {
            k_order_init<<<(unsigned)vpet_ceil_div(ORDER_BUCKETS, 256), 256, 0, s>>>(p.xmm, p.xhist);
            VPET_LAUNCH_CHECK();
            const unsigned gb = (unsigned)vpet_ceil_div(L.N, 256);
            k_order_features<<<gb, 256, 0, s>>>(sc[i].x, L.N, sc[i].ldx, L.L, W, p.xfeat, p.xmm);
            VPET_LAUNCH_CHECK();
            k_order_hist<<<gb, 256, 0, s>>>(p.xfeat, p.xmm, L.N, L.nlev, tu.pilot_stride, p.xhist);
            VPET_LAUNCH_CHECK();
            k_order_scan_sums<<<SCAN_BLOCKS, 1024, 0, s>>>(p.xhist, p.xhist + ORDER_BUCKETS);
            k_order_scan_top<<<1, 1024, 0, s>>>(p.xhist + ORDER_BUCKETS);
            k_order_scan<<<SCAN_BLOCKS, 1024, 0, s>>>(p.xhist, p.xhist + ORDER_BUCKETS);
            VPET_LAUNCH_CHECK();
            k_order_scatter<<<gb, 256, 0, s>>>(p.xfeat, p.xmm, L.N, L.nlev, tu.pilot_stride, p.xhist, p.xperm);
            VPET_LAUNCH_CHECK();
        }
        k_pack_x<<<(unsigned)vpet_ceil_div(L.Np, 8 * PACK_ROWS), 256, 0, s>>>(sc[i].x, L.N, L.Np, sc[i].ldx, L.L, L.Kp,
                                                                           mode, W, p.mu, L.G,
                                                                           xorder ? p.xperm : nullptr, p.B, p.fx,
                                                                           p.xs, L.ldxs);
        VPET_LAUNCH_CHECK();
        if (xorder) {
            k_tile_boxes<<<(unsigned)vpet_ceil_div(L.nt64, 8), 256, 0, s>>>(p.fx, L.N, L.nt64, p.tbox);
            VPET_LAUNCH_CHECK();
        }
    }
    // work order: costliest scans first (longest-processing-time round robin)
    int order[MAX_ITEMS];
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int a = 1; a < n; ++a) {
        const int v = order[a];
        const double cv = (double)BL.lay[v].Jp * (double)BL.lay[v].N;
        int b = a;
        while (b > 0 && (double)BL.lay[order[b - 1]].Jp * (double)BL.lay[order[b - 1]].N < cv) {
            order[b] = order[b - 1];
            --b;
        }
        order[b] = v;
    }
    // draw-tile width of the pass being set up: the tuning's, except for top-r pilot levels, which
    // run 64-draw tiles (their key rows leave room for two CTAs per SM only there)
    int pass_bn = tu.bn;
    auto fill_item = [&](ItemTc& I, int i, int64_t stride, int kt, int lim, const float* thr0) -> int {
        const Layout& L = BL.lay[i];
        const Ptrs& p = ptr[i];
        int r;
        if ((r = make_tmap(&I.tmA, p.A, L.Jp, L.Kp, BM, 1))) return r;
        const int64_t Nn = L.N / stride;
        // the draw operand holds G copies of Np rows (one per centring group); a pilot's strided
        // view takes every stride-th row of all of them (Np is a multiple of the stride)
        if ((r = make_tmap(&I.tmB, p.B, stride == 1 ? (int64_t)L.G * L.Np : (int64_t)L.G * L.Np / stride, L.Kp,
                           pass_bn, stride)))
            return r;
        (void)Nn;
        I.J = L.J;
        I.N = stride == 1 ? L.N : Nn;
        I.keys = p.keys;
        I.idx = p.idx;
        I.cnt = p.cnt;
        I.thr = p.thr;
        I.thr0 = thr0;
        I.ntiles = (int)vpet_ceil_div(I.N, pass_bn);
        I.C = L.C;
        // with 128-draw tiles two epilogue threads serve a voxel, each with its own
        // half-list that keeps its own kt smallest and receives half of every tile;
        // with 64-draw tiles one thread uses the whole list (half 1 stays empty)
        const bool halves = pass_bn == 128;
        I.C2 = halves ? L.C / 2 : L.C;
        I.hstride = (int)L.Jp;
        I.kt = kt;
        const int per_tile = halves ? pass_bn / 2 : pass_bn;
        const int cap = kt + (kt / 4 > 64 ? kt / 4 : 64);
        I.cap = cap < I.C2 ? cap : I.C2;
        // a half-list may grow to the whole list's limit (its capacity allows it): halving
        // the limit would double a pilot's compactions
        I.lim = lim < I.C2 ? lim : I.C2;
        I.lim0 = 2 * kt + per_tile < I.lim ? 2 * kt + per_tile : I.lim;
        return ABC_OK;
    };
    int maxlev = 0;
    for (int i = 0; i < n; ++i) maxlev = BL.lay[i].nlev > maxlev ? BL.lay[i].nlev : maxlev;
    if (dump) maxlev = 0;
    // draw tiles a pass can skip, from the thresholds in thr0 (needs the ordered draws)
    // with_thr: the pass has thresholds in thr0 (else every tile is kept); order: nearest first
    auto keep_tiles = [&](int i, int64_t npass, unsigned long long* tally, bool with_thr, bool order) -> int {
        const Layout& L = BL.lay[i];
        KeepArgs K;
        memset(&K, 0, sizeof K);
        K.fy = ptr[i].fy;
        K.thr0 = with_thr ? ptr[i].thr0 : nullptr;
        K.order = order ? 1 : 0;
        K.ynorm = ptr[i].ynorm;
        K.tbox = ptr[i].tbox;
        K.ktile = ptr[i].ktile;
        K.kcount = ptr[i].kcount;
        K.tally = tally;
        K.J = L.J;
        K.N = npass;
        K.nt64 = L.nt64;
        for (int l = 0; l < L.L; ++l) K.Wc[(3 * l) / L.L] += sc[i].w[l];
        K.cE = error_coef(L);
        K.split = mode != ABC_FP32;
        K.sc = split_coef(L);
        K.c0 = ptr[i].c0;
        K.dn = ptr[i].dn;
        K.bn = pass_bn;
        k_keep_tiles<<<(unsigned)L.nvt, 256, 0, s>>>(K);
        VPET_LAUNCH_CHECK();
        return ABC_OK;
    };
    // pilot passes, coarsest level first; pilot level lv reads the leading
    // ceil(N / stride) packed draws (the draws j with j % stride == 0)
    for (int lv = maxlev - 1; lv >= 0; --lv) {
        memset(&T, 0, sizeof T);
        memset(&PB, 0, sizeof PB);
        int m = 0, mp = 0;
        // a level whose ranks are all small runs as top-r pilots (one kernel variant per launch)
        bool lev_topr = true;
        for (int i = 0; i < n; ++i)
            if (BL.lay[i].nlev > lv && BL.lay[i].lev_rank[lv] > TOPR_MAX) lev_topr = false;
        pass_bn = lev_topr ? 64 : tu.bn;
        for (int oi = 0; oi < n; ++oi) {
            const int i = order[oi];
            const Layout& L = BL.lay[i];
            if (L.nlev <= lv) continue;
            const int r = L.lev_rank[lv];
            const int lim = (int)(4 * (int64_t)r + 256 < L.C ? 4 * (int64_t)r + 256 : L.C);
            const bool has_thr = lv + 1 < L.nlev;
            if ((rc = fill_item(T.item[m], i, 1, r, lim, has_thr ? ptr[i].thr0 : nullptr))) return rc;
            T.tgroup[m] = L.G > 1 ? ptr[i].tgroup : nullptr;
            T.grows[m] = L.Np;
            const int64_t npass = vpet_ceil_div(L.N, L.lev_stride[lv]);
            T.item[m].N = npass;
            T.item[m].ntiles = (int)vpet_ceil_div(npass, pass_bn);
            // the pass's draw tiles nearest first (all of them at the coarsest level, which has no
            // threshold yet): the pilot's kept keys settle early (its result does not depend on the order)
            if ((rc = keep_tiles(i, npass, nullptr, has_thr, true))) return rc;
            T.item[m].ktile = ptr[i].ktile;
            T.item[m].kcount = ptr[i].kcount;
            T.item[m].kstride = L.nt64;
            T.vt_prefix[m + 1] = T.vt_prefix[m] + L.Jp / BM;
            // the finest split-form pilot reports its rank-rk key, which k_need_threshold turns
            // into the voxel's need threshold for the main pass
            const int rsel = (lv == 0 && L.rk > 0) ? L.rk : r;
            if (lev_topr) {
                // small rank: the kernel keeps each voxel's r smallest keys itself and
                // writes the threshold; no lists, no selection pass
                T.item[m].rsel = r;
                T.item[m].rk = lv == 0 ? L.rk : 0;
                T.item[m].thr_out = ptr[i].thr0;
            } else {
                PB.item[mp] = PilotItem{ptr[i].keys, ptr[i].cnt, ptr[i].thr0, L.J, L.C, rsel, pass_bn == 128 ? L.C / 2 : L.C, L.Jp};
                PB.v_prefix[mp + 1] = PB.v_prefix[mp] + L.J;
                ++mp;
            }
            ++m;
        }
        T.n_items = m;
        T.status = status;
        T.counter = counters + (lv + 1);
        T.wait_ns = g_wait_ns;
        T.withhold = g_withhold;
        PB.n_items = mp;
        PB.status = status;
        if ((rc = dispatch_tc<false>(nkb, pass_bn, T, tu.ctas_per_sm, s, lev_topr))) return rc;
        if (mp > 0) {
            k_pilot_threshold<<<(unsigned)vpet_ceil_div(PB.v_prefix[mp], 8), 256, 0, s>>>(PB);
            VPET_LAUNCH_CHECK();
        }
        if (lv == 0 && mode != ABC_FP32) {
            BatchNeed NB;
            memset(&NB, 0, sizeof NB);
            int mn = 0;
            for (int i = 0; i < n; ++i) {
                const Layout& L = BL.lay[i];
                if (L.nlev <= 0) continue;
                NB.item[mn] = NeedItem{ptr[i].thr0, ptr[i].ynorm, ptr[i].c0, ptr[i].dn, L.J, split_coef(L)};
                NB.v_prefix[mn + 1] = NB.v_prefix[mn] + L.J;
                ++mn;
            }
            NB.n_items = mn;
            if (mn > 0) {
                k_need_threshold<<<(unsigned)vpet_ceil_div(NB.v_prefix[mn], 256), 256, 0, s>>>(NB);
                VPET_LAUNCH_CHECK();
            }
        }
    }
    pass_bn = tu.bn;
    // draw tiles the main pass can skip (needs the pilot thresholds and the ordered draws)
    unsigned long long* tally = (unsigned long long*)(wsb + 192);
    bool skip[MAX_ITEMS];
    for (int i = 0; i < n; ++i) {
        const Layout& L = BL.lay[i];
        skip[i] = dump == nullptr && L.nlev > 0 && L.N > 1;
        if (skip[i] && (rc = keep_tiles(i, L.N, tally, true, false))) return rc;
    }
    // main pass
    memset(&T, 0, sizeof T);
    for (int oi = 0; oi < n; ++oi) {
        const int i = order[oi];
        const Layout& L = BL.lay[i];
        if ((rc = fill_item(T.item[oi], i, 1, L.kt, L.C, L.nlev > 0 ? ptr[i].thr0 : nullptr))) return rc;
        T.tgroup[oi] = L.G > 1 ? ptr[i].tgroup : nullptr;
        T.grows[oi] = L.Np;
        if (skip[i]) {
            T.item[oi].ktile = ptr[i].ktile;
            T.item[oi].kcount = ptr[i].kcount;
            T.item[oi].kstride = L.nt64;
        }
        T.vt_prefix[oi + 1] = T.vt_prefix[oi] + L.Jp / BM;
    }
    T.n_items = n;
    T.status = status;
    T.counter = counters;
    T.dump = dump;
    T.ld_dump = ld_dump;
    T.wait_ns = g_wait_ns;
    T.withhold = g_withhold;
    if (dump) return dispatch_tc<true>(nkb, 128, T, tu.ctas_per_sm, s);
    if (g_prof_start) VPET_CUDA(record_event(g_prof_start, s));
    if ((rc = dispatch_tc<false>(nkb, tu.bn, T, tu.ctas_per_sm, s))) return rc;
    if (g_prof_stop) VPET_CUDA(record_event(g_prof_stop, s));
    // finalize
    memset(&F, 0, sizeof F);
    int sortcap = 64;
    for (int i = 0; i < n; ++i) {
        const Layout& L = BL.lay[i];
        FinItem& f = F.item[i];
        f.J = L.J;
        f.N = L.N;
        f.L = L.L;
        f.k = L.k;
        f.C = L.C;
        f.C2 = tu.bn == 128 ? L.C / 2 : L.C;
        f.hstride = L.Jp;
        f.kt = L.kt;
        f.mode = mode;
        f.sortcap = L.sortcap;
        f.cacc = split_coef(L).cacc;
        f.y = sc[i].y;
        f.ldy = sc[i].ldy;
        f.x = sc[i].x;
        f.ldx = sc[i].ldx;
        f.ynorm = ptr[i].ynorm;
        f.c0 = ptr[i].c0;
        f.dn = ptr[i].dn;
        f.perm = (dump == nullptr && L.J > 1) ? ptr[i].perm : nullptr;
        f.xperm = (dump == nullptr && L.N > 1) ? ptr[i].xperm : nullptr;
        f.xs = ptr[i].xs;
        f.ldxs = L.ldxs;
        f.tbox = (dump == nullptr && L.N > 1) ? ptr[i].tbox : nullptr;
        f.fy = ptr[i].fy;
        f.nt64 = L.nt64;
        for (int l = 0; l < L.L; ++l) f.Wc[(3 * l) / L.L] += sc[i].w[l];
        f.keys = ptr[i].keys;
        f.idx = ptr[i].idx;
        f.cnt = ptr[i].cnt;
        f.thr = ptr[i].thr;
        f.out_idx = sc[i].idx;
        f.out_dist = sc[i].dist;
        f.w = ptr[i].wdev;
        if (L.rcap > 0 && dump == nullptr) {
            f.rq_rows = ptr[i].rrow;
            f.rq_thr = ptr[i].rthr;
            f.rq_dk = ptr[i].rthr + L.rcapa;
            f.rq_count = ptr[i].rq;
            f.rq_cap = queue_cap(L);
        }
        F.v_prefix[i + 1] = F.v_prefix[i] + L.J;
        if (L.sortcap > sortcap) sortcap = L.sortcap;
    }
    F.n_items = n;
    F.sortcap = sortcap;
    F.status = status;
    F.force_rescue = g_force_rescue;
    int warps = 8;
    while (warps > 1 && (size_t)warps * sortcap * 8 > 64 * 1024) warps >>= 1;
    const size_t fsmem = (size_t)warps * (1024 + 2 * MAXL * 4 + (size_t)sortcap * 8);
    static size_t fin_configured_dev[64] = {};
    int fdev = 0;
    VPET_CUDA(cudaGetDevice(&fdev));
    VPET_ARG(fdev >= 0 && fdev < 64, "device ordinal %d out of range", fdev);
    if (fsmem > 48 * 1024 && fsmem > fin_configured_dev[fdev]) {
        VPET_CUDA(cudaFuncSetAttribute(k_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
        fin_configured_dev[fdev] = fsmem;
    }
    k_finalize<<<(unsigned)vpet_ceil_div(F.v_prefix[n], warps), warps * 32, fsmem, s>>>(F);
    VPET_LAUNCH_CHECK();
    if (mode == ABC_FP32 || dump != nullptr) return ABC_OK;

    // rescue pass of the split form: the voxels the finalize queued, each with the exact
    // threshold its net's k-th distance asks for, go through the fused kernel once more
    // (their candidate lists rebuilt in their own rows) and a second finalize.  Queue
    // lengths stay on the device: positions past them are skipped.
    BatchRescue RB;
    memset(&RB, 0, sizeof RB);
    for (int i = 0; i < n; ++i) {
        const Layout& L = BL.lay[i];
        const Ptrs& p = ptr[i];
        RB.item[i] = RescueItem{p.rq,   p.rrow, p.rthr, p.rthr + L.rcapa, p.rrow2, p.rthr2, p.rdk2,
                                p.rtg,  queue_cap(L), L.Jg, L.J, L.G, L.Kp, p.A, p.RA,
                                L.lrows * (int64_t)L.C, L.Cr};
    }
    RB.n_items = n;
    k_rescue_count<<<(unsigned)num_sms() * 2, 256, 0, s>>>(RB);
    VPET_LAUNCH_CHECK();
    k_rescue_layout<<<(unsigned)n, 256, 0, s>>>(RB);
    VPET_LAUNCH_CHECK();
    k_rescue_place<<<(unsigned)num_sms() * 4, 256, 0, s>>>(RB);
    VPET_LAUNCH_CHECK();
    memset(&T, 0, sizeof T);
    for (int oi = 0; oi < n; ++oi) {
        const int i = order[oi];
        const Layout& L = BL.lay[i];
        const Ptrs& p = ptr[i];
        const bool xorder = L.N > 1;
        if (xorder) {
            KeepArgs K;
            memset(&K, 0, sizeof K);
            K.fy = p.fy;
            K.thr0 = p.rthr2;
            K.ynorm = p.ynorm;
            K.tbox = p.tbox;
            K.ktile = p.ktile;
            K.kcount = p.kcount;
            K.J = L.rcapa;
            K.N = L.N;
            K.nt64 = L.nt64;
            for (int l = 0; l < L.L; ++l) K.Wc[(3 * l) / L.L] += sc[i].w[l];
            K.cE = error_coef(L);
            K.split = 1;
            K.sc = split_coef(L);
            K.c0 = p.c0;
            K.dn = p.dn;
            K.rows = p.rrow2;
            K.count = p.rq + 1;
            K.bn = tu.bn;
            k_keep_tiles<<<(unsigned)(L.rcapa / BM), 256, 0, s>>>(K);
            VPET_LAUNCH_CHECK();
        }
        if ((rc = fill_item(T.item[oi], i, 1, L.kt, L.C, p.rthr2))) return rc;
        if ((rc = make_tmap(&T.item[oi].tmA, p.RA, L.rcapa, L.Kp, BM, 1))) return rc;
        T.item[oi].J = L.rcapa;
        T.item[oi].rows = p.rrow2;
        // lists by queue position, Cr entries each (shared, atomically appended: no compaction)
        T.item[oi].C = L.Cr;
        T.item[oi].C2 = tu.bn == 128 ? L.Cr / 2 : L.Cr;
        T.item[oi].cnt = p.rcnt;
        T.item[oi].thr = p.rthrh;
        T.item[oi].hstride = (int)L.rcapa;
        T.tgroup[oi] = L.G > 1 ? p.rtg : nullptr;   // each rescue tile lies in one centring group
        T.grows[oi] = L.Np;
        if (xorder) {
            T.item[oi].ktile = p.ktile;
            T.item[oi].kcount = p.kcount;
            T.item[oi].kstride = L.nt64;
        }
        T.dyn_count[oi] = p.rq + 1;
        T.dyn_C[oi] = p.rq + 2 + 3 * L.G + 1;
        T.vt_prefix[oi + 1] = T.vt_prefix[oi] + L.rcapa / BM * RESCUE_SEGMENTS;
    }
    T.nseg = RESCUE_SEGMENTS;
    T.n_items = n;
    T.status = status;
    T.counter = counters + (MAX_PILOT_LEVELS + 1);
    T.wait_ns = g_wait_ns;
    T.withhold = g_withhold;
    if ((rc = dispatch_tc<false>(nkb, tu.bn, T, tu.ctas_per_sm, s))) return rc;
    for (int i = 0; i < n; ++i) {
        FinItem& f = F.item[i];
        const Layout& L = BL.lay[i];
        f.rows = ptr[i].rrow2;
        f.rcount = ptr[i].rq + 1;
        f.C = L.Cr;                                  // lists by queue position
        f.C2 = tu.bn == 128 ? L.Cr / 2 : L.Cr;
        f.cnt = ptr[i].rcnt;
        f.thr = ptr[i].rthrh;
        f.hstride = L.rcapa;
        f.dyn_C = ptr[i].rq + 2 + 3 * L.G + 1;
        f.rq_rows = nullptr;
        f.rq_thr = nullptr;
        f.rq_dk = ptr[i].rdk2;   // read by the rescue finalize
        f.rq_count = nullptr;
        f.rq_cap = 0;
        F.v_prefix[i + 1] = F.v_prefix[i] + L.rcapa;
    }
    k_finalize<<<(unsigned)vpet_ceil_div(F.v_prefix[n], warps), warps * 32, fsmem, s>>>(F);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

bool g_has_default = false;   // abc_set_default_tuning was called
Tuning g_default_tuning = default_tuning(ABC_BF16_RESCORE);

Tuning tuning_for(int mode) { return g_has_default ? g_default_tuning : default_tuning(mode); }
Tuning tuning_for(int mode, int L, int k) {
    return g_has_default ? g_default_tuning : default_tuning_for_shape(mode, L, k);
}

ScanSpec single(const float* y, int64_t J, int ldy, const float* x, int64_t N, int ldx, int L, const float* w, int k,
                int32_t* idx, float* dist) {
    return ScanSpec{y, J, ldy, x, N, ldx, L, w, k, idx, dist};
}

int to_tuning(const abc_tuning* t, int mode, Tuning* out) {
    if (!t) {
        *out = tuning_for(mode);
        return ABC_OK;
    }
    *out = Tuning{t->bn, t->ctas_per_sm, t->pilot_stride, t->pilot_factor};
    return check_tuning(*out);
}

int gather_scans(const abc_scan* scans, int n, ScanSpec* out) {
    VPET_ARG(scans, "batch: null scan array");
    VPET_ARG(n >= 1 && n <= MAX_ITEMS, "batch: 1..%d scans per call (got %d)", MAX_ITEMS, n);
    for (int i = 0; i < n; ++i) {
        const abc_scan& c = scans[i];
        out[i] = ScanSpec{c.y_dev, c.J, c.ldy, c.x_dev, c.N, c.ldx, c.L, c.w_host, c.k, c.idx_dev, c.dist_dev};
    }
    return ABC_OK;
}

}  // namespace

namespace vpet {

size_t topk_workspace_bytes(int64_t J, int64_t N, int L, int k, int precision) {
    ScanSpec c = single(nullptr, J, L, nullptr, N, L, L, nullptr, k, nullptr, nullptr);
    BatchLayout* B = new BatchLayout;
    make_batch_layout(&c, 1, precision, tuning_for(precision, L, k), B);
    const size_t t = B->total;
    delete B;
    return t;
}

int topk_on_workspace(const float* y, int64_t J, int ldy, const float* x, int64_t N, int ldx, int L, const float* w,
                      int k, int precision, void* ws, size_t ws_bytes, int32_t* idx, float* dist, cudaStream_t s) {
    const ScanSpec c = single(y, J, ldy, x, N, ldx, L, w, k, idx, dist);
    return run_batch(&c, 1, precision, tuning_for(precision, L, k), ws, ws_bytes, nullptr, 0, s);
}

}  // namespace vpet

extern "C" size_t abc_workspace_size(int64_t J, int64_t N, int32_t L, int32_t k, int32_t precision) {
    if (J < 1 || N < 1 || L < 1 || L > 61 || k < 1 || k > N || k > 2048) return 0;
    if (precision != ABC_FP32 && precision != ABC_BF16_RESCORE && precision != ABC_SPLIT_DRAWS) return 0;
    return vpet::topk_workspace_bytes(J, N, L, k, precision);
}

extern "C" int abc_discrepancy_topk(const float* y_dev, int64_t J, int32_t ldy, const float* x_dev, int64_t N,
                                    int32_t ldx, int32_t L, const float* w_host, int32_t k, int32_t precision,
                                    void* workspace, size_t ws_bytes, int32_t* idx_dev, float* dist_dev, void* stream) {
    vpet::clear_error();
    return vpet::topk_on_workspace(y_dev, J, ldy, x_dev, N, ldx, L, w_host, k, precision, workspace, ws_bytes, idx_dev,
                                   dist_dev, (cudaStream_t)stream);
}

extern "C" int abc_topk_work(const void* workspace, int64_t out_host[2], void* stream) {
    vpet::clear_error();
    VPET_ARG(workspace && out_host, "abc_topk_work: null pointer");
    unsigned long long t[2];
    VPET_CUDA(cudaMemcpyAsync(t, (const uint8_t*)workspace + 192, sizeof t, cudaMemcpyDeviceToHost,
                              (cudaStream_t)stream));
    VPET_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    out_host[0] = (int64_t)t[0];
    out_host[1] = (int64_t)t[1];
    return ABC_OK;
}

extern "C" int abc_default_tuning(int32_t precision, abc_tuning* out) {
    vpet::clear_error();
    VPET_ARG(out, "abc_default_tuning: null pointer");
    VPET_ARG(precision == ABC_FP32 || precision == ABC_BF16_RESCORE || precision == ABC_SPLIT_DRAWS,
             "abc_default_tuning: unknown precision");
    const Tuning t = tuning_for(precision);
    out->bn = t.bn;
    out->ctas_per_sm = t.ctas_per_sm;
    out->pilot_stride = t.pilot_stride;
    out->pilot_factor = t.pilot_factor;
    return ABC_OK;
}

extern "C" int abc_set_default_tuning(const abc_tuning* t) {
    vpet::clear_error();
    Tuning tu;
    const int rc = to_tuning(t, ABC_BF16_RESCORE, &tu);
    if (rc) return rc;
    g_has_default = t != nullptr;
    if (t) g_default_tuning = tu;
    return ABC_OK;
}

extern "C" size_t abc_batch_workspace_size(const abc_scan* scans, int32_t n_scans, int32_t precision) {
    ScanSpec sp[MAX_ITEMS];
    if (!scans || n_scans < 1 || n_scans > MAX_ITEMS) return 0;
    if (precision != ABC_FP32 && precision != ABC_BF16_RESCORE && precision != ABC_SPLIT_DRAWS) return 0;
    for (int i = 0; i < n_scans; ++i) {
        const abc_scan& c = scans[i];
        if (c.J < 1 || c.N < 1 || c.L < 1 || c.L > 61 || c.k < 1 || c.k > c.N || c.k > 2048) return 0;
        sp[i] = ScanSpec{c.y_dev, c.J, c.ldy, c.x_dev, c.N, c.ldx, c.L, c.w_host, c.k, c.idx_dev, c.dist_dev};
    }
    BatchLayout* B = new BatchLayout;
    make_batch_layout(sp, n_scans, precision, tuning_for(precision), B);
    const size_t t = B->total;
    delete B;
    return t;
}

extern "C" int abc_batch_discrepancy_topk(const abc_scan* scans, int32_t n_scans, int32_t precision,
                                          const abc_tuning* tuning, void* workspace, size_t ws_bytes, void* stream) {
    vpet::clear_error();
    ScanSpec sp[MAX_ITEMS];
    int rc = gather_scans(scans, n_scans, sp);
    if (rc) return rc;
    Tuning tu;
    if ((rc = to_tuning(tuning, precision, &tu))) return rc;
    return run_batch(sp, n_scans, precision, tu, workspace, ws_bytes, nullptr, 0, (cudaStream_t)stream);
}

extern "C" int abc_debug_inject_stall(int64_t withheld_tile, uint64_t wait_ns) {
    vpet::clear_error();
    VPET_ARG(wait_ns == 0 || (wait_ns >= 1000000ull && wait_ns <= 10000000000ull),
             "abc_debug_inject_stall: wait_ns must be 0 (default) or in [1 ms, 10 s]");
    g_withhold = withheld_tile < 0 ? -1 : withheld_tile;
    g_wait_ns = wait_ns == 0 ? WAIT_NS_DEFAULT : wait_ns;
    return ABC_OK;
}

extern "C" int abc_debug_order(int32_t mode) {
    vpet::clear_error();
    VPET_ARG(mode >= 0 && mode <= 2, "abc_debug_order: mode must be 0, 1 or 2 (got %d)", mode);
    g_order_mode = mode;
    return ABC_OK;
}

extern "C" int abc_debug_force_rescue(int32_t mode) {
    vpet::clear_error();
    VPET_ARG(mode >= 0 && mode <= 7, "abc_debug_force_rescue: mode is a mask of 1, 2 and 4 (got %d)", mode);
    g_force_rescue = mode;
    return ABC_OK;
}

extern "C" int abc_profile_events(void* start_event, void* stop_event) {
    vpet::clear_error();
    VPET_ARG((start_event == nullptr) == (stop_event == nullptr), "abc_profile_events: give both events or neither");
    g_prof_start = (cudaEvent_t)start_event;
    g_prof_stop = (cudaEvent_t)stop_event;
    return ABC_OK;
}

extern "C" int abc_topk_status(const void* workspace, int32_t status_host[8], void* stream) {
    vpet::clear_error();
    VPET_ARG(workspace && status_host, "abc_topk_status: null pointer");
    int32_t st[8];
    VPET_CUDA(cudaMemcpyAsync(st, workspace, sizeof st, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    VPET_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    for (int i = 0; i < 8; ++i) status_host[i] = st[i];
    return ABC_OK;
}

// Test hook: the raw tensor-core keys d' for every (voxel, draw) pair, written to
// dump_dev (Jp x Np, row stride ld_dump >= Np) without the top-k.
extern "C" int abc_debug_gemm_keys(const float* y_dev, int64_t J, int32_t ldy, const float* x_dev, int64_t N,
                                   int32_t ldx, int32_t L, const float* w_host, int32_t precision, void* workspace,
                                   size_t ws_bytes, float* dump_dev, int64_t ld_dump, void* stream) {
    vpet::clear_error();
    VPET_ARG(dump_dev && ld_dump >= vpet_round_up(N, 128), "abc_debug_gemm_keys: dump too small");
    const ScanSpec c = single(y_dev, J, ldy, x_dev, N, ldx, L, w_host, 1, nullptr, nullptr);
    return run_batch(&c, 1, precision, tuning_for(precision), workspace, ws_bytes, dump_dev, ld_dump,
                     (cudaStream_t)stream);
}

namespace vpet {
long long launches();
}

extern "C" int abc_launch_info(int64_t* grid, int32_t* resident_per_sm, int64_t* kernel_launches) {
    vpet::clear_error();
    VPET_ARG(grid && resident_per_sm && kernel_launches, "abc_launch_info: null pointer");
    *grid = g_last_grid;
    *resident_per_sm = g_last_resident;
    *kernel_launches = vpet::launches();
    return ABC_OK;
}
