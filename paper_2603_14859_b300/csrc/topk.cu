// Discrepancy + top-k (Algorithm 1, steps 4-5) on the 5th-generation tensor
// cores, fused so the J x N distance matrix never reaches memory.
//
// d_jn = sum_l w_l (y_jl - x_nl)^2 = ||yh_j||^2 + ||xh_n||^2 - 2 yh_j . xh_n with
// yh = sqrt(w)(y - mu), xh = sqrt(w)(x - mu) (mu = mean voxel TAC; distances
// are translation invariant).  The ranking key d' = ||xh||^2 - 2 yh . xh is one
// GEMM: voxel rows A = [yh .., 1, 1, 1], draw rows B = [-2 xh .., n_hi, n_mid, n_lo]
// where n = ||xh||^2 is split over three bf16 columns.
//   ABC_FP32:  yh, xh split into bf16 hi + lo; A = [yh_hi, yh_hi, yh_lo, 1,1,1],
//              B = [-2xh_hi, -2xh_lo, -2xh_hi, n_hi, n_mid, n_lo]: three bf16
//              products per term, |error| <= E(voxel) (bound below).
//   ABC_BF16_RESCORE: one bf16 product per term.
//
// Kernel `k_tc_topk`: one CTA owns 128 voxels (one TMEM lane each) and streams
// every draw tile of 128 rows through shared memory (TMA, 128-byte swizzle).
// Warp roles: 0 = TMA producer, 1 = TMEM allocator + MMA issuer (one thread),
// 2..5 = epilogue (thread <-> voxel).  Accumulators are double-buffered in TMEM
// (2 x 128 fp32 columns) so MMA of tile t+1 overlaps the epilogue of tile t.
// The epilogue reads 32 columns at a time and takes their minimum; a thread
// whose minimum is within its voxel's running threshold stages the 32 keys in
// shared memory, and the warp then appends each such voxel's passing
// (key, draw index) pairs to that voxel's candidate list in global memory with
// one coalesced store.  When a list could overflow, the warp compacts it
// (radix select of the kt-th key, in-place filtering) and tightens the
// threshold, so each list always holds every draw whose key is at most the
// kt-th smallest seen (the "net": kt = 2k for ABC_FP32, 4k for ABC_BF16_RESCORE).
//
// Pilot passes of the same kernel over every 16th (then 256th, ...) draw (a
// strided TMA tensor map) first find each voxel's r-th smallest key,
// r = 1.5 kt / 16; as draws are i.i.d. within each model, about 1.5 kt of all N
// draws fall below it, so the main pass starts from that threshold, appends
// ~1.5 kt candidates per voxel and normally never compacts.  Each pilot starts
// from the next coarser pilot's threshold in the same way.  Nothing relies on
// the prediction for correctness: a list always holds every draw below its
// voxel's threshold.
//
// Kernel `k_finalize` (one warp per voxel) re-scores the net exactly as
// sum_l w_l (y_l - x_l)^2 in fp32, selects the exact k-th distance d_k, and
// certifies the result: with E bounding |computed d' - exact d'| for any draw
// that could beat d_k (its ||xh|| <= ||yh|| + sqrt(d_k)), every draw outside
// the net has computed key > T_out, so none can beat d_k when
// T_out >= d_k - ||yh||^2 + E.  ABC_FP32 resolves an uncertified voxel by an
// exact fp32 scan of all draws, which makes its accepted set the exact fp32
// top-k; ABC_BF16_RESCORE counts uncertified voxels (abc_topk_status).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "common.cuh"
#include "select.cuh"
#include "tc_ptx.cuh"

using namespace vpet;

namespace {

constexpr int BM = 128;          // voxels per CTA = TMEM lanes
constexpr int BN = 128;          // draws per tile = accumulator columns
constexpr int KBLK = 64;         // bf16 per K-block (128-byte rows)
constexpr int KBLK_BYTES = BM * KBLK * 2;   // 16 KB (BM == BN)
constexpr int TC_THREADS = 192;
constexpr uint64_t WAIT_NS = 2000000000ull; // 2 s bound on any barrier wait
constexpr int MAXL = 64;
constexpr int PILOT_STRIDE = 16;
constexpr int MAX_PILOT_LEVELS = 4;

struct Weights {
    float w[MAXL];
    float sw[MAXL];   // sqrt(w)
};

struct Layout {
    int mode;          // ABC_FP32 / ABC_BF16_RESCORE
    int L, k, Kp, nkb, C, kt, cap, sortcap;
    int nlev;                          // pilot levels (finest first)
    int lev_rank[4];
    int64_t lev_stride[4];
    int64_t J, N, Jp, Np;
    int npart;
    size_t off_mu, off_part, off_ynorm, off_a, off_b, off_keys, off_idx, off_cnt, off_thr, off_thr0, off_status, total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

Layout make_layout(int64_t J, int64_t N, int L, int k, int mode) {
    Layout s;
    memset(&s, 0, sizeof s);
    s.mode = mode;
    s.L = L;
    s.k = k;
    s.J = J;
    s.N = N;
    const int kcols = mode == ABC_FP32 ? 3 * L + 3 : L + 3;
    s.Kp = (int)vpet_round_up(kcols, KBLK);
    s.nkb = s.Kp / KBLK;
    const int64_t net = (int64_t)(mode == ABC_FP32 ? 2 : 4) * k;
    s.kt = (int)(net < N ? net : N);
    s.cap = s.kt + (s.kt / 4 > 64 ? s.kt / 4 : 64);
    // pilot: the r-th smallest key over every 16th draw predicts the 1.5 kt-th
    // smallest over all draws (draws are i.i.d. within each model)
    // Levels of pilots: level i uses every 16^i-th draw and a target rank
    // r_i = ceil(f r_{i-1} / 16), r_0 = kt; each starts from the next coarser
    // level's threshold.  f = 1.5 predicts 1.5 r_{i-1} draws below the
    // threshold at the finer level; for a small r_i the rank statistic is noisy
    // (relative sd ~ 1 / sqrt(r_i)), so f grows until an under-prediction is
    // more than ~4 sd away.
    s.nlev = 0;
    int64_t rr = s.kt, stride = 1;
    while (s.nlev < MAX_PILOT_LEVELS) {
        int64_t r_next = (3 * rr + 31) / 32;
        for (int it = 0; it < 8; ++it) {
            const double f = (double)r_next * PILOT_STRIDE / (double)rr;       // predicted count / needed
            if (1.0 - 1.0 / f >= 4.0 / sqrt((double)r_next)) break;
            r_next = r_next + r_next / 2 + 1;
        }
        const int64_t n_next = N / (stride * PILOT_STRIDE);
        if (n_next < 8 * r_next || n_next < 4 * BN) break;
        stride *= PILOT_STRIDE;
        rr = r_next;
        s.lev_rank[s.nlev] = (int)rr;
        s.lev_stride[s.nlev] = stride;
        s.nlev++;
    }
    s.C = (int)vpet_round_up(3 * (int64_t)s.kt + 2 * BN, 32);
    s.sortcap = next_pow2(k + 8);     // k plus a few ties at the k-th distance
    if (s.sortcap < 64) s.sortcap = 64;
    s.Jp = vpet_round_up(J > 0 ? J : 1, BM);
    s.Np = vpet_round_up(N > 0 ? N : 1, BN);
    s.npart = (int)(vpet_ceil_div(J, 256) < 1024 ? vpet_ceil_div(J, 256) : 1024);
    if (s.npart < 1) s.npart = 1;
    size_t o = 0;
    s.off_status = o; o = align256(o + 64 * sizeof(int32_t));
    s.off_mu = o; o = align256(o + MAXL * sizeof(float));
    s.off_part = o; o = align256(o + (size_t)s.npart * MAXL * sizeof(float));
    s.off_ynorm = o; o = align256(o + (size_t)s.Jp * sizeof(float));
    s.off_a = o; o = align256(o + (size_t)s.Jp * s.Kp * 2);
    s.off_b = o; o = align256(o + (size_t)s.Np * s.Kp * 2);
    s.off_keys = o; o = align256(o + (size_t)J * s.C * sizeof(float));
    s.off_idx = o; o = align256(o + (size_t)J * s.C * sizeof(int32_t));
    s.off_cnt = o; o = align256(o + (size_t)s.Jp * sizeof(int32_t));
    s.off_thr = o; o = align256(o + (size_t)s.Jp * sizeof(float));
    s.off_thr0 = o; o = align256(o + (size_t)s.Jp * sizeof(float));
    s.total = o;
    return s;
}

// ------------------------------------------------------------------ packing
// Column mean of y over voxels, deterministic two-stage reduction.
__global__ void k_colmean_part(const float* __restrict__ y, int64_t J, int ldy, int L, float* __restrict__ part,
                               int npart) {
    __shared__ float red[4][MAXL];
    const int l = threadIdx.x & 63, g = threadIdx.x >> 6;
    const int64_t per = (J + npart - 1) / npart;
    const int64_t j0 = blockIdx.x * per, j1 = j0 + per < J ? j0 + per : J;
    float s = 0.0f;
    if (l < L)
        for (int64_t j = j0 + g; j < j1; j += 4) s += y[j * ldy + l];
    red[g][l] = s;
    __syncthreads();
    if (g == 0) part[(size_t)blockIdx.x * MAXL + l] = red[0][l] + red[1][l] + red[2][l] + red[3][l];
}

__global__ void k_colmean_final(const float* __restrict__ part, int npart, int64_t J, float* __restrict__ mu) {
    const int l = threadIdx.x;
    double s = 0.0;
    for (int b = 0; b < npart; ++b) s += part[(size_t)b * MAXL + l];
    mu[l] = (float)(s / (double)J);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ __nv_bfloat16 bf(float v) { return __float2bfloat16_rn(v); }

// One warp per voxel row: A row of the GEMM and ||yh||^2.
__global__ void k_pack_y(const float* __restrict__ y, int64_t J, int64_t Jp, int ldy, int L, int Kp, int mode,
                         Weights W, const float* __restrict__ mu, __nv_bfloat16* __restrict__ A,
                         float* __restrict__ ynorm) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= Jp) return;
    __nv_bfloat16* row = A + j * Kp;
    if (j >= J) {
        for (int e = lane; e < Kp; e += 32) row[e] = bf(0.0f);
        if (lane == 0) ynorm[j] = 0.0f;
        return;
    }
    const float* yr = y + j * ldy;
    float ss = 0.0f;
    for (int l = lane; l < L; l += 32) {
        const float v = W.sw[l] * (yr[l] - mu[l]);
        ss = fmaf(v, v, ss);
    }
    ss = warp_sum(ss);
    if (lane == 0) ynorm[j] = ss;
    for (int e = lane; e < Kp; e += 32) {
        float out = 0.0f;
        if (mode == ABC_FP32) {
            if (e < 3 * L) {
                const int l = e % L;
                const float v = W.sw[l] * (yr[l] - mu[l]);
                const float hi = __bfloat162float(bf(v));
                out = e < 2 * L ? hi : v - hi;
            } else if (e < 3 * L + 3) {
                out = 1.0f;
            }
        } else {
            if (e < L) out = W.sw[e] * (yr[e] - mu[e]);
            else if (e < L + 3) out = 1.0f;
        }
        row[e] = bf(out);
    }
}

// One warp per draw row: B row of the GEMM.
__global__ void k_pack_x(const float* __restrict__ x, int64_t N, int64_t Np, int ldx, int L, int Kp, int mode,
                         Weights W, const float* __restrict__ mu, __nv_bfloat16* __restrict__ B) {
    const int lane = threadIdx.x & 31;
    const int64_t n = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (n >= Np) return;
    __nv_bfloat16* row = B + n * Kp;
    if (n >= N) {
        for (int e = lane; e < Kp; e += 32) row[e] = bf(0.0f);
        return;
    }
    const float* xr = x + n * ldx;
    float ss = 0.0f;
    for (int l = lane; l < L; l += 32) {
        float v = W.sw[l] * (xr[l] - mu[l]);
        if (mode != ABC_FP32) v = __bfloat162float(bf(v));   // norm of the rounded vector
        ss = fmaf(v, v, ss);
    }
    ss = warp_sum(ss);
    const float n1 = __bfloat162float(bf(ss));
    const float r1 = ss - n1;
    const float n2 = __bfloat162float(bf(r1));
    const float n3 = r1 - n2;
    const int aug = mode == ABC_FP32 ? 3 * L : L;
    for (int e = lane; e < Kp; e += 32) {
        float out = 0.0f;
        if (e < aug) {
            const int l = e % L;
            const float v = W.sw[l] * (xr[l] - mu[l]);
            const float hi = __bfloat162float(bf(v));
            if (mode == ABC_FP32) out = -2.0f * ((e >= L && e < 2 * L) ? (v - hi) : hi);
            else out = -2.0f * hi;
        } else if (e == aug) {
            out = n1;
        } else if (e == aug + 1) {
            out = n2;
        } else if (e == aug + 2) {
            out = n3;
        }
        row[e] = bf(out);
    }
}

// ------------------------------------------------------------------ fused GEMM + filter
struct TcParams {
    int64_t J, N;
    int ntiles, C, kt, cap;
    int lim;                     // a list is compacted once it could exceed lim entries (lim <= C)
    float* keys;
    int32_t* idx;
    int32_t* cnt;
    float* thr;                  // final running threshold per voxel
    const float* thr0;           // initial threshold per voxel (pilot), or null = +huge
    int32_t* status;
    float* dump;                 // debug probe: raw keys, Jp x Np (nullptr in production)
    int64_t ld_dump;
};

constexpr int STAGE_LD = 36;     // floats per staged row (16-byte aligned, conflict-free)

// Bound on |computed d' - exact d'| for any draw with ||xh|| <= R.
__device__ __forceinline__ float err_bound(float cE, float ry, float R) { return cE * (2.0f * ry * R + R * R); }

// Tightens voxel j's candidate list to the keys <= its kt-th key; returns the new
// threshold and updates cnt.
__device__ __forceinline__ float compact_list(const TcParams& P, int64_t j, int& cnt, uint32_t* hist, int lane) {
    float* kj = P.keys + j * P.C;
    int32_t* ij = P.idx + j * P.C;
    const uint32_t T = warp_select(kj, cnt, P.kt - 1, 3, hist, lane);
    const int q = warp_compact(kj, ij, cnt, T, P.cap, lane);
    cnt = q < P.cap ? q : P.cap;
    if (q > P.cap && lane == 0) atomicOr(&P.cnt[j], 0x40000000);   // overflow: resolved by an exact scan
    return key2f(T);
}

__device__ __forceinline__ float min32(const float (&v)[32]) {
    float m[11];
#pragma unroll
    for (int i = 0; i < 10; ++i) asm("min.f32 %0, %1, %2, %3;" : "=f"(m[i]) : "f"(v[3 * i]), "f"(v[3 * i + 1]), "f"(v[3 * i + 2]));
    m[10] = fminf(v[30], v[31]);
    float a, b, c, d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(a) : "f"(m[0]), "f"(m[1]), "f"(m[2]));
    asm("min.f32 %0, %1, %2, %3;" : "=f"(b) : "f"(m[3]), "f"(m[4]), "f"(m[5]));
    asm("min.f32 %0, %1, %2, %3;" : "=f"(c) : "f"(m[6]), "f"(m[7]), "f"(m[8]));
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(m[9]), "f"(m[10]), "f"(a));
    return fminf(fminf(b, c), d);
}

// One 32-column chunk of the epilogue: filter, then warp-cooperative appends.
__device__ __forceinline__ void epilogue_chunk(const TcParams& P, float (&v)[32], int64_t n0, int64_t jbase,
                                               float thr, int& cnt, float* stage, int lane) {
    if (n0 + 32 > P.N) {
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (n0 + i >= P.N) v[i] = __int_as_float(0x7F800000);   // +inf: never kept
    }
    const bool slow = min32(v) <= thr;
    uint32_t bal = __ballot_sync(0xFFFFFFFFu, slow);
    if (!bal) return;
    if (slow) {
        float4* dst = (float4*)(stage + lane * STAGE_LD);
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    __syncwarp();
    const uint32_t lt = (1u << lane) - 1u;
    while (bal) {
        const int s = __ffs(bal) - 1;
        bal &= bal - 1;
        const float val = stage[s * STAGE_LD + lane];
        const float ts = __shfl_sync(0xFFFFFFFFu, thr, s);
        const int cs = __shfl_sync(0xFFFFFFFFu, cnt, s);
        const bool pass = val <= ts;
        const uint32_t pb = __ballot_sync(0xFFFFFFFFu, pass);
        if (pass) {
            const int64_t at = (jbase + s) * (int64_t)P.C + cs + __popc(pb & lt);
            P.keys[at] = val;
            P.idx[at] = (int32_t)(n0 + lane);
        }
        if (lane == s) cnt += __popc(pb);
    }
    __syncwarp();
}

template <int NKB, int STAGES, bool DUMP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_topk(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams P) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                                        // NKB x 16 KB
    uint8_t* sB = smem + NKB * KBLK_BYTES;                     // STAGES x NKB x 16 KB
    float* sStage = (float*)(sB + STAGES * NKB * KBLK_BYTES);  // 4 warps x 32 x STAGE_LD
    uint32_t* hist = (uint32_t*)(sStage + 4 * 32 * STAGE_LD);  // 4 warps x 256
    uint64_t* bars = (uint64_t*)(hist + 4 * 256);
    uint64_t* full = bars;                  // [STAGES]
    uint64_t* empty = bars + STAGES;        // [STAGES]
    uint64_t* tfull = bars + 2 * STAGES;    // [2]
    uint64_t* tempty = bars + 2 * STAGES + 2;
    uint64_t* afull = bars + 2 * STAGES + 4;
    uint32_t* tmem_holder = (uint32_t*)(bars + 2 * STAGES + 5);
    volatile int* s_err = (volatile int*)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.x * BM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(ptx::smem_u32(&full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(ptx::smem_u32(&tfull[a]), 1);
            ptx::mbar_init(ptx::smem_u32(&tempty[a]), 4);
        }
        ptx::mbar_init(ptx::smem_u32(afull), 1);
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
    const int ntiles = P.ntiles;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            ptx::tma_prefetch_desc(&tmA);
            ptx::tma_prefetch_desc(&tmB);
            const uint32_t ab = ptx::smem_u32(afull);
            ptx::mbar_arrive_expect_tx(ab, NKB * KBLK_BYTES);
            for (int kb = 0; kb < NKB; ++kb)
                ptx::tma_load_2d(ptx::smem_u32(sA + kb * KBLK_BYTES), &tmA, ab, kb * KBLK, (int32_t)m0);
            for (int t = 0; t < ntiles; ++t) {
                const int s = t % STAGES;
                const uint32_t ph = (uint32_t)(t / STAGES) & 1u;
                if (!ptx::mbar_wait(ptx::smem_u32(&empty[s]), ph ^ 1u, WAIT_NS)) { *s_err = 1; break; }
                if (*s_err) break;
                const uint32_t fb = ptx::smem_u32(&full[s]);
                ptx::mbar_arrive_expect_tx(fb, NKB * KBLK_BYTES);
                for (int kb = 0; kb < NKB; ++kb)
                    ptx::tma_load_2d(ptx::smem_u32(sB + (s * NKB + kb) * KBLK_BYTES), &tmB, fb, kb * KBLK, t * BN);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (single thread)
        if (lane == 0) {
            constexpr uint32_t idesc = ptx::idesc_bf16_f32(BM, BN);
            bool ok = ptx::mbar_wait(ptx::smem_u32(afull), 0, WAIT_NS);
            if (!ok) *s_err = 1;
            const uint32_t a_base = ptx::smem_u32(sA);
            for (int t = 0; ok && t < ntiles; ++t) {
                const int s = t % STAGES;
                const uint32_t ph = (uint32_t)(t / STAGES) & 1u;
                const int acc = t & 1;
                const uint32_t aph = (uint32_t)(t >> 1) & 1u;
                if (!ptx::mbar_wait(ptx::smem_u32(&tempty[acc]), aph ^ 1u, WAIT_NS) ||
                    !ptx::mbar_wait(ptx::smem_u32(&full[s]), ph, WAIT_NS)) {
                    *s_err = 1;
                    break;
                }
                if (*s_err) break;
                ptx::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc * BN);
                const uint32_t b_base = ptx::smem_u32(sB + s * NKB * KBLK_BYTES);
#pragma unroll
                for (int kb = 0; kb < NKB; ++kb) {
#pragma unroll
                    for (int kk = 0; kk < KBLK / 16; ++kk) {
                        const uint64_t ad = ptx::desc_sw128(a_base + kb * KBLK_BYTES + kk * 32);
                        const uint64_t bd = ptx::desc_sw128(b_base + kb * KBLK_BYTES + kk * 32);
                        ptx::mma_bf16(d_tmem, ad, bd, idesc, (kb | kk) ? 1u : 0u);
                    }
                }
                ptx::mma_commit(ptx::smem_u32(&empty[s]));
                ptx::mma_commit(ptx::smem_u32(&tfull[acc]));
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, thread <-> voxel
        const int q = warp & 3;                          // TMEM lane quadrant of this warp
        const int row = q * 32 + lane;
        const int64_t jbase = m0 + q * 32;
        const int64_t j = jbase + lane;
        const bool valid = j < P.J;
        uint32_t* whist = hist + (warp - 2) * 256;
        float* stage = sStage + (warp - 2) * 32 * STAGE_LD;
        float thr = valid ? (P.thr0 ? P.thr0[j] : 3.0e38f) : -3.0e38f;
        int cnt = 0;
        for (int t = 0; t < ntiles; ++t) {
            const int acc = t & 1;
            const uint32_t aph = (uint32_t)(t >> 1) & 1u;
            if (!ptx::mbar_wait(ptx::smem_u32(&tfull[acc]), aph, WAIT_NS)) { *s_err = 1; }
            if (__any_sync(0xFFFFFFFFu, *s_err != 0)) break;
            ptx::tc_fence_after();
            const int64_t nbase = (int64_t)t * BN;
#pragma unroll 1
            for (int h = 0; h < BN / 64; ++h) {
                uint32_t r0[32], r1[32];
                const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + h * 64);
                ptx::tmem_ld32_async(ta, r0);
                ptx::tmem_ld32_async(ta + 32, r1);
                ptx::tmem_wait_ld();
                ptx::tmem_fence_regs(r0);
                ptx::tmem_fence_regs(r1);
                float v0[32], v1[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) { v0[i] = __uint_as_float(r0[i]); v1[i] = __uint_as_float(r1[i]); }
                if (DUMP) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        P.dump[(m0 + row) * P.ld_dump + nbase + h * 64 + i] = v0[i];
                        P.dump[(m0 + row) * P.ld_dump + nbase + h * 64 + 32 + i] = v1[i];
                    }
                    continue;
                }
                epilogue_chunk(P, v0, nbase + h * 64, jbase, thr, cnt, stage, lane);
                epilogue_chunk(P, v1, nbase + h * 64 + 32, jbase, thr, cnt, stage, lane);
            }
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&tempty[acc]));
            if (DUMP) continue;
            // compaction of lists that might not fit the next tile
            uint32_t need = __ballot_sync(0xFFFFFFFFu, valid && cnt > P.lim - BN);
            while (need) {
                const int src = __ffs(need) - 1;
                need &= need - 1;
                int c2 = __shfl_sync(0xFFFFFFFFu, cnt, src);
                const float nt = compact_list(P, jbase + src, c2, whist, lane);
                if (lane == src) {
                    cnt = c2;
                    thr = nt;
                }
            }
        }
        if (valid && !DUMP) {
            atomicOr(&P.cnt[j], cnt);      // cnt[] was zeroed; keeps the overflow bit
            P.thr[j] = thr;
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
// list is emptied for the main pass.
__global__ void k_pilot_threshold(float* keys, int32_t* cnt, int C, int r, int64_t J, float* thr0) {
    __shared__ uint32_t hist[8][256];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + wid;
    if (j >= J) return;
    const int c = cnt[j] & 0x3FFFFFFF;
    float t = 3.0e38f;
    if (!(cnt[j] & 0x40000000) && c >= r) t = key2f(warp_select(keys + j * C, c, r - 1, 3, hist[wid], lane));
    if (lane == 0) {
        thr0[j] = t;
        cnt[j] = 0;
    }
}

// ------------------------------------------------------------------ finalize
struct FinParams {
    int64_t J, N;
    int L, k, C, kt, mode, sortcap;
    float cE;
    const float* y;
    int ldy;
    const float* x;
    int ldx;
    const float* ynorm;
    float* keys;
    int32_t* idx;
    int32_t* cnt;
    const float* thr;
    int32_t* status;
    int32_t* out_idx;
    float* out_dist;
};

// Exact fp32 distance sum_l w_l (y_l - x_l)^2 in a fixed order (y in shared memory).
__device__ __forceinline__ float exact_dist(const float* ys, const float* x, int L, const Weights& W) {
    const float4* xr = (const float4*)x;
    float d = 0.0f;
    int l = 0;
    for (; l + 4 <= L; l += 4) {
        const float4 xv = __ldg(xr + (l >> 2));
        const float e0 = ys[l] - xv.x, e1 = ys[l + 1] - xv.y, e2 = ys[l + 2] - xv.z, e3 = ys[l + 3] - xv.w;
        d = fmaf(W.w[l] * e0, e0, d);
        d = fmaf(W.w[l + 1] * e1, e1, d);
        d = fmaf(W.w[l + 2] * e2, e2, d);
        d = fmaf(W.w[l + 3] * e3, e3, d);
    }
    for (; l < L; ++l) {
        const float e = ys[l] - x[l];
        d = fmaf(W.w[l] * e, e, d);
    }
    return d;
}

// exact_dist for two rows at once (same operation order), loads interleaved.
__device__ __forceinline__ void exact_dist2(const float* ys, const float* xa, const float* xb, int L, const Weights& W,
                                            float& da, float& db) {
    const float4* ra = (const float4*)xa;
    const float4* rb = (const float4*)xb;
    float a = 0.0f, b = 0.0f;
    int l = 0;
    for (; l + 4 <= L; l += 4) {
        const float4 va = __ldg(ra + (l >> 2));
        const float4 vb = __ldg(rb + (l >> 2));
        float e = ys[l] - va.x;
        a = fmaf(W.w[l] * e, e, a);
        e = ys[l + 1] - va.y;
        a = fmaf(W.w[l + 1] * e, e, a);
        e = ys[l + 2] - va.z;
        a = fmaf(W.w[l + 2] * e, e, a);
        e = ys[l + 3] - va.w;
        a = fmaf(W.w[l + 3] * e, e, a);
        e = ys[l] - vb.x;
        b = fmaf(W.w[l] * e, e, b);
        e = ys[l + 1] - vb.y;
        b = fmaf(W.w[l + 1] * e, e, b);
        e = ys[l + 2] - vb.z;
        b = fmaf(W.w[l + 2] * e, e, b);
        e = ys[l + 3] - vb.w;
        b = fmaf(W.w[l + 3] * e, e, b);
    }
    for (; l < L; ++l) {
        float e = ys[l] - xa[l];
        a = fmaf(W.w[l] * e, e, a);
        e = ys[l] - xb[l];
        b = fmaf(W.w[l] * e, e, b);
    }
    da = a;
    db = b;
}

// status[1]: voxels resolved by the exact scan; [2]: tie overflow; [3]: uncertified (bf16 mode)
__global__ void k_finalize(FinParams P, Weights W) {
    extern __shared__ __align__(16) uint8_t fsm[];
    const int warps = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* hist = (uint32_t*)fsm + wid * 256;
    float* ys = (float*)(fsm + warps * 1024) + wid * MAXL;
    unsigned long long* sbuf = (unsigned long long*)(fsm + warps * 1024 + warps * MAXL * 4) + (size_t)wid * P.sortcap;
    const int64_t j = (int64_t)blockIdx.x * warps + wid;
    if (j >= P.J) return;
    float* kj = P.keys + j * P.C;
    int32_t* ij = P.idx + j * P.C;
    const int raw = P.cnt[j];
    int cnt = raw & 0x3FFFFFFF;
    for (int l = lane; l < P.L; l += 32) ys[l] = P.y[j * P.ldy + l];
    __syncwarp();
    bool scan = (raw & 0x40000000) != 0;
    uint32_t K = 0;
    if (!scan) {
        // 1. the net: every draw outside it has computed key > T_out
        float T_out = P.thr[j];
        if (P.mode != ABC_FP32 && cnt > P.kt) {
            const uint32_t T = warp_select(kj, cnt, P.kt - 1, 3, hist, lane);
            cnt = warp_compact(kj, ij, cnt, T, P.C, lane);
            T_out = key2f(T);
        }
        // 2. exact fp32 re-score of the net (two candidates per lane in flight)
        int i = lane;
        for (; i + 32 < cnt; i += 64) {
            const int32_t n0 = ij[i], n1 = ij[i + 32];
            float d0, d1;
            exact_dist2(ys, P.x + (int64_t)n0 * P.ldx, P.x + (int64_t)n1 * P.ldx, P.L, W, d0, d1);
            kj[i] = d0;
            kj[i + 32] = d1;
        }
        if (i < cnt) kj[i] = exact_dist(ys, P.x + (int64_t)ij[i] * P.ldx, P.L, W);
        __syncwarp();
        // 3. exact k-th distance and the certificate
        bool cert = false;
        if (cnt >= P.k) {
            K = warp_select(kj, cnt, P.k - 1, 4, hist, lane);
            const float dk = key2f(K);
            const float yn = P.ynorm[j];
            const float slack = 4.0f * (float)P.L * 0x1p-24f;
            const float ry = sqrtf(yn);
            const float R = ry + sqrtf(dk * (1.0f + slack)) + 1e-30f;
            const float need = dk * (1.0f + slack) - yn * (1.0f - slack) + err_bound(P.cE, ry, R);
            cert = T_out >= 2.9e38f || T_out >= need;
        }
        if (!cert) {
            if (P.mode == ABC_FP32) scan = true;
            else if (lane == 0) atomicAdd(&P.status[3], 1);
        }
        if (!scan && cnt < P.k) K = 0xFFFFFFFFu;
    }
    if (scan) {
        // exact fp32 scan of every draw (candidate list rebuilt with exact keys)
        if (lane == 0) atomicAdd(&P.status[1], 1);
        cnt = 0;
        float thr = __int_as_float(0x7F800000);
        for (int64_t base = 0; base < P.N; base += 32) {
            const int64_t n = base + lane;
            const float d = n < P.N ? exact_dist(ys, P.x + n * P.ldx, P.L, W) : __int_as_float(0x7F800000);
            const bool take = n < P.N && d <= thr;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, take);
            if (take) {
                const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                kj[pos] = d;
                ij[pos] = (int32_t)n;
            }
            cnt += __popc(bal);
            if (cnt > P.C - 32) {
                __syncwarp();
                const uint32_t T = warp_select(kj, cnt, P.k - 1, 4, hist, lane);
                const int q = warp_compact(kj, ij, cnt, T, P.C - 64, lane);
                cnt = q < P.C - 64 ? q : P.C - 64;
                thr = key2f(T);
            }
        }
        __syncwarp();
        K = cnt >= P.k ? warp_select(kj, cnt, P.k - 1, 4, hist, lane) : 0xFFFFFFFFu;
    }
    // 4. keep everything at or below the exact k-th distance, sort by (distance, index)
    if (cnt > P.k) {
        const int g = warp_compact(kj, ij, cnt, K, P.sortcap, lane);
        if (g > P.sortcap && lane == 0) atomicAdd(&P.status[2], 1);
        cnt = g < P.sortcap ? g : P.sortcap;
    }
    int n2 = 32;
    while (n2 < cnt) n2 <<= 1;
    for (int i = lane; i < n2; i += 32)
        sbuf[i] = i < cnt ? (((unsigned long long)f2key(kj[i]) << 32) | (uint32_t)ij[i]) : ~0ull;
    warp_bitonic_sort(sbuf, n2, lane);
    for (int r = lane; r < P.k; r += 32) {
        const unsigned long long e = r < cnt ? sbuf[r] : ~0ull;
        P.out_idx[j * P.k + r] = r < cnt ? (int32_t)(uint32_t)e : -1;
        P.out_dist[j * P.k + r] = r < cnt ? key2f((uint32_t)(e >> 32)) : __int_as_float(0x7F800000);
    }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
cudaEvent_t g_prof_start = nullptr, g_prof_stop = nullptr;

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

int make_tmap(CUtensorMap* m, void* base, int64_t rows, int Kp, int row_step = 1) {
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2 * row_step};
    const cuuint32_t box[2] = {(cuuint32_t)KBLK, (cuuint32_t)BM};
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

template <int NKB>
constexpr int stages_for() { return NKB == 1 ? 4 : (NKB == 2 ? 4 : 3); }

template <int NKB>
size_t tc_smem_bytes() {
    return 1024 + (size_t)NKB * KBLK_BYTES * (1 + stages_for<NKB>()) + 4 * 32 * STAGE_LD * 4 + 4 * 256 * 4 +
           (2 * stages_for<NKB>() + 8) * 8;
}

template <int NKB, bool DUMP>
int launch_tc(const CUtensorMap& ta, const CUtensorMap& tb, const TcParams& P, int64_t grid, cudaStream_t s) {
    constexpr int S = stages_for<NKB>();
    const size_t smem = tc_smem_bytes<NKB>();
    static bool configured = false;
    if (!configured) {
        VPET_CUDA(cudaFuncSetAttribute(k_tc_topk<NKB, S, DUMP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    k_tc_topk<NKB, S, DUMP><<<(unsigned)grid, TC_THREADS, smem, s>>>(ta, tb, P);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

template <bool DUMP>
int dispatch_tc(int nkb, const CUtensorMap& ta, const CUtensorMap& tb, const TcParams& P, int64_t grid,
                cudaStream_t s) {
    switch (nkb) {
        case 1: return launch_tc<1, DUMP>(ta, tb, P, grid, s);
        case 2: return launch_tc<2, DUMP>(ta, tb, P, grid, s);
        case 3: return launch_tc<3, DUMP>(ta, tb, P, grid, s);
        default:
            vpet::set_error("unsupported K-block count %d", nkb);
            return ABC_ERR_UNSUPPORTED;
    }
}

float error_coef(const Layout& lay) {
    // |d' error| <= cE (2 ||yh|| R + R^2) for a draw with ||xh|| <= R.
    //  ABC_FP32: bf16 hi + lo of each operand leaves |a - a_hi - a_lo| <= 2^-16 |a|,
    //   |a_lo| <= 2^-8 |a|, so the three products miss at most 3 * 2^-16 |a b|;
    //  ABC_BF16_RESCORE: one rounding of each operand and of the norm, 2^-8 each.
    // Both add fp32 accumulation over Kp terms, the fp32 norm and the fp32
    // centring / scaling of the operands.
    const float split = lay.mode == ABC_FP32 ? 3.0f * 0x1p-16f : 3.0f * 0x1p-8f;
    return split + (float)(3 * lay.Kp + lay.L + 16) * 0x1p-24f;
}

int validate(const float* y, int64_t J, int ldy, const float* x, int64_t N, int ldx, int L, const float* w, int k,
             int mode) {
    VPET_ARG(J >= 1 && N >= 1, "abc_discrepancy_topk: J and N must be >= 1");
    VPET_ARG(N < ((int64_t)1 << 31), "abc_discrepancy_topk: N must be < 2^31");
    VPET_ARG(L >= 1 && L <= 61, "abc_discrepancy_topk: L must be in 1..61 (got %d)", L);
    VPET_ARG(k >= 1 && k <= 2048 && k <= N, "abc_discrepancy_topk: need 1 <= k <= min(N, 2048)");
    VPET_ARG(mode == ABC_FP32 || mode == ABC_BF16_RESCORE, "abc_discrepancy_topk: unknown precision %d", mode);
    VPET_ARG(y && x && w, "abc_discrepancy_topk: null pointer");
    VPET_ARG(ldy >= L && ldx >= L && ldx % 4 == 0 && ldy % 4 == 0,
             "abc_discrepancy_topk: ldy, ldx must be >= L and multiples of 4");
    VPET_ARG(((uintptr_t)y & 15) == 0 && ((uintptr_t)x & 15) == 0, "abc_discrepancy_topk: y, x must be 16-byte aligned");
    bool any = false;
    for (int l = 0; l < L; ++l) {
        VPET_ARG(w[l] >= 0.0f && w[l] == w[l], "abc_discrepancy_topk: weights must be >= 0");
        any |= w[l] > 0.0f;
    }
    VPET_ARG(any, "abc_discrepancy_topk: all weights are zero");
    return ABC_OK;
}

int run_topk(const float* y, int64_t J, int ldy, const float* x, int64_t N, int ldx, int L, const float* w, int k,
             int mode, void* ws, size_t ws_bytes, int32_t* out_idx, float* out_dist, float* dump, int64_t ld_dump,
             cudaStream_t s) {
    const Layout lay = make_layout(J, N, L, k, mode);
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < lay.total) {
        vpet::set_error("abc_discrepancy_topk: workspace needs %zu bytes, 256-aligned (got %zu)", lay.total, ws_bytes);
        return ABC_ERR_WORKSPACE;
    }
    if (!dump) VPET_ARG(out_idx && out_dist, "abc_discrepancy_topk: null output");
    int rc = get_encoder();
    if (rc) return rc;
    uint8_t* base = (uint8_t*)ws;
    float* mu = (float*)(base + lay.off_mu);
    float* part = (float*)(base + lay.off_part);
    float* ynorm = (float*)(base + lay.off_ynorm);
    __nv_bfloat16* A = (__nv_bfloat16*)(base + lay.off_a);
    __nv_bfloat16* B = (__nv_bfloat16*)(base + lay.off_b);
    int32_t* status = (int32_t*)(base + lay.off_status);
    int32_t* cnt = (int32_t*)(base + lay.off_cnt);
    Weights W;
    memset(&W, 0, sizeof W);
    for (int l = 0; l < L; ++l) {
        W.w[l] = w[l];
        W.sw[l] = sqrtf(w[l]);
    }
    VPET_CUDA(cudaMemsetAsync(status, 0, 64 * sizeof(int32_t), s));
    VPET_CUDA(cudaMemsetAsync(cnt, 0, (size_t)lay.Jp * sizeof(int32_t), s));
    k_colmean_part<<<lay.npart, 256, 0, s>>>(y, J, ldy, L, part, lay.npart);
    VPET_LAUNCH_CHECK();
    k_colmean_final<<<1, MAXL, 0, s>>>(part, lay.npart, J, mu);
    VPET_LAUNCH_CHECK();
    k_pack_y<<<(unsigned)vpet_ceil_div(lay.Jp, 8), 256, 0, s>>>(y, J, lay.Jp, ldy, L, lay.Kp, mode, W, mu, A, ynorm);
    VPET_LAUNCH_CHECK();
    k_pack_x<<<(unsigned)vpet_ceil_div(lay.Np, 8), 256, 0, s>>>(x, N, lay.Np, ldx, L, lay.Kp, mode, W, mu, B);
    VPET_LAUNCH_CHECK();
    CUtensorMap ta, tb;
    if ((rc = make_tmap(&ta, A, lay.Jp, lay.Kp))) return rc;
    if ((rc = make_tmap(&tb, B, lay.Np, lay.Kp))) return rc;
    TcParams P;
    P.J = J;
    P.N = N;
    P.ntiles = (int)(lay.Np / BN);
    P.C = lay.C;
    P.lim = lay.C;
    P.kt = lay.kt;
    P.cap = lay.cap;
    P.keys = (float*)(base + lay.off_keys);
    P.idx = (int32_t*)(base + lay.off_idx);
    P.cnt = cnt;
    P.thr = (float*)(base + lay.off_thr);
    P.status = status;
    P.dump = dump;
    P.ld_dump = ld_dump;
    const int64_t grid = lay.Jp / BM;
    if (dump) return dispatch_tc<true>(lay.nkb, ta, tb, P, grid, s);
    P.thr0 = nullptr;
    float* thr0 = (float*)(base + lay.off_thr0);
    for (int lv = lay.nlev - 1; lv >= 0; --lv) {
        // pilot pass over every lev_stride-th draw (strided tensor map, no copy)
        const int64_t st = lay.lev_stride[lv];
        const int64_t Ns = N / st;
        const int r = lay.lev_rank[lv];
        CUtensorMap tp;
        if ((rc = make_tmap(&tp, B, Ns, lay.Kp, (int)st))) return rc;
        TcParams Q = P;
        Q.N = Ns;
        Q.ntiles = (int)vpet_ceil_div(Ns, BN);
        Q.kt = r;
        Q.cap = r + (r / 4 > 64 ? r / 4 : 64);
        Q.lim = (int)(4 * (int64_t)r + 2 * BN < lay.C ? 4 * (int64_t)r + 2 * BN : lay.C);
        if ((rc = dispatch_tc<false>(lay.nkb, ta, tp, Q, grid, s))) return rc;
        k_pilot_threshold<<<(unsigned)vpet_ceil_div(J, 8), 256, 0, s>>>(P.keys, cnt, lay.C, r, J, thr0);
        VPET_LAUNCH_CHECK();
        P.thr0 = thr0;
    }
    if (g_prof_start) VPET_CUDA(cudaEventRecord(g_prof_start, s));
    if ((rc = dispatch_tc<false>(lay.nkb, ta, tb, P, grid, s))) return rc;
    if (g_prof_stop) VPET_CUDA(cudaEventRecord(g_prof_stop, s));
    FinParams F;
    F.J = J;
    F.N = N;
    F.L = L;
    F.k = k;
    F.C = lay.C;
    F.kt = lay.kt;
    F.mode = mode;
    F.sortcap = lay.sortcap;
    F.cE = error_coef(lay);
    F.y = y;
    F.ldy = ldy;
    F.x = x;
    F.ldx = ldx;
    F.ynorm = ynorm;
    F.keys = P.keys;
    F.idx = P.idx;
    F.cnt = cnt;
    F.thr = P.thr;
    F.status = status;
    F.out_idx = out_idx;
    F.out_dist = out_dist;
    int warps = 8;
    while (warps > 1 && (size_t)warps * lay.sortcap * 8 > 64 * 1024) warps >>= 1;
    const size_t fsmem = (size_t)warps * (1024 + MAXL * 4 + (size_t)lay.sortcap * 8);
    static size_t fin_configured = 0;
    if (fsmem > 48 * 1024 && fsmem > fin_configured) {
        VPET_CUDA(cudaFuncSetAttribute(k_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
        fin_configured = fsmem;
    }
    k_finalize<<<(unsigned)vpet_ceil_div(J, warps), warps * 32, fsmem, s>>>(F, W);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

}  // namespace

namespace vpet {

size_t topk_workspace_bytes(int64_t J, int64_t N, int L, int k, int precision) {
    return make_layout(J, N, L, k, precision).total;
}

int topk_on_workspace(const float* y, int64_t J, int ldy, const float* x, int64_t N, int ldx, int L, const float* w,
                      int k, int precision, void* ws, size_t ws_bytes, int32_t* idx, float* dist, cudaStream_t s) {
    const int rc = validate(y, J, ldy, x, N, ldx, L, w, k, precision);
    if (rc) return rc;
    return run_topk(y, J, ldy, x, N, ldx, L, w, k, precision, ws, ws_bytes, idx, dist, nullptr, 0, s);
}

}  // namespace vpet

extern "C" size_t abc_workspace_size(int64_t J, int64_t N, int32_t L, int32_t k, int32_t precision) {
    if (J < 1 || N < 1 || L < 1 || L > 61 || k < 1 || k > N || k > 2048) return 0;
    if (precision != ABC_FP32 && precision != ABC_BF16_RESCORE) return 0;
    return make_layout(J, N, L, k, precision).total;
}

extern "C" int abc_discrepancy_topk(const float* y_dev, int64_t J, int32_t ldy, const float* x_dev, int64_t N,
                                    int32_t ldx, int32_t L, const float* w_host, int32_t k, int32_t precision,
                                    void* workspace, size_t ws_bytes, int32_t* idx_dev, float* dist_dev, void* stream) {
    vpet::clear_error();
    const int rc = validate(y_dev, J, ldy, x_dev, N, ldx, L, w_host, k, precision);
    if (rc) return rc;
    return run_topk(y_dev, J, ldy, x_dev, N, ldx, L, w_host, k, precision, workspace, ws_bytes, idx_dev, dist_dev,
                    nullptr, 0, (cudaStream_t)stream);
}

extern "C" int abc_profile_events(void* start_event, void* stop_event) {
    vpet::clear_error();
    VPET_ARG((start_event == nullptr) == (stop_event == nullptr), "abc_profile_events: give both events or neither");
    g_prof_start = (cudaEvent_t)start_event;
    g_prof_stop = (cudaEvent_t)stop_event;
    return ABC_OK;
}

extern "C" int abc_topk_status(const void* workspace, int32_t status_host[4], void* stream) {
    vpet::clear_error();
    VPET_ARG(workspace && status_host, "abc_topk_status: null pointer");
    int32_t st[4];
    VPET_CUDA(cudaMemcpyAsync(st, workspace, sizeof st, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    VPET_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    status_host[0] = st[0];
    status_host[1] = st[1];
    status_host[2] = st[2];
    status_host[3] = st[3];
    return ABC_OK;
}

// Test hook: the raw tensor-core keys d' for every (voxel, draw) pair, written to
// dump_dev (Jp x Np, row stride ld_dump >= Np) without the top-k.
extern "C" int abc_debug_gemm_keys(const float* y_dev, int64_t J, int32_t ldy, const float* x_dev, int64_t N,
                                   int32_t ldx, int32_t L, const float* w_host, int32_t precision, void* workspace,
                                   size_t ws_bytes, float* dump_dev, int64_t ld_dump, void* stream) {
    vpet::clear_error();
    const int rc = validate(y_dev, J, ldy, x_dev, N, ldx, L, w_host, 1, precision);
    if (rc) return rc;
    VPET_ARG(dump_dev && ld_dump >= vpet_round_up(N, BN), "abc_debug_gemm_keys: dump too small");
    return run_topk(y_dev, J, ldy, x_dev, N, ldx, L, w_host, 1, precision, workspace, ws_bytes, nullptr, nullptr,
                    dump_dev, ld_dump, (cudaStream_t)stream);
}
