// Top-k by the frame-weighted L1 distance d(y, x) = sum_l w_l |y_l - x_l|, the
// distance Sec. V recommends (Algorithm 1, steps 4-5 with rho = L1).  The L1
// distance has no inner-product expansion, so there is no tensor-core form: a
// block of voxels (four per warp) walks the draws in shared-memory tiles, every
// lane accumulating eight draws' distances to each of its warp's four voxels in
// fp32 over the frames in order (each draw value read once serves four), and
// appends the draws at or below its voxel's running threshold to the voxel's
// candidate list; a list near its capacity is cut to its k smallest (exact
// radix select), which sets the threshold.  With few voxels the draws are split
// into segments scanned by separate blocks (one list per voxel and segment).  A
// second kernel joins a voxel's lists, selects and sorts the final k by
// (distance, draw index).
#include <string.h>

#include "common.cuh"
#include "select.cuh"

namespace {

using vpet::f2key;
using vpet::key2f;

constexpr int L1_TILE = 256;            // draws per shared-memory tile (8 per lane)
constexpr int L1_TS = L1_TILE + 2;      // padded row of the transposed tile (8-byte aligned; few bank conflicts)
constexpr int L1_MAXL = 64;

struct L1Args {
    const float* y;
    int64_t J;
    int ldy;
    const float* x;
    int64_t N;
    int ldx;
    int L, k, C;                        // frames, accepted draws, list capacity per voxel and segment
    int S;                              // draw segments (blockIdx.y): lists per voxel
    int64_t seg_len;                    // draws per segment (a multiple of the tile)
    float w[L1_MAXL];
    float* keys;                        // J x S x C candidate distances
    int32_t* idx;                       // J x S x C candidate draw indices
    int32_t* cnt;                       // J x S list lengths
    int32_t* status;                    // [0] voxels whose ties at a cut exceeded the list
    float* out_dist;
    int32_t* out_idx;
    int sortcap;
};

// Cuts a list (in increasing draw order) to its entries <= T, T its exact k-th key,
// keeping at most cap: when more entries tie at T than fit, the ties with the lowest
// draw indices stay and later draws must be strictly below T.  Returns the new
// threshold; cnt becomes the new length.
__device__ float cut_list(float* kj, int32_t* ij, int& cnt, int k, int cap, uint32_t* hist, int lane,
                          int32_t* status) {
    const uint32_t T = vpet::warp_select(kj, cnt, k - 1, 4, hist, lane);
    const vpet::KthKey c = vpet::warp_count_key(kj, cnt, T, lane);
    if (c.n_less + c.n_eq <= cap) {
        cnt = vpet::warp_compact(kj, ij, cnt, T, cap, lane);
        return key2f(T);
    }
    const uint32_t Ti = vpet::warp_select_tie_index(kj, ij, cnt, T, cap - c.n_less - 1, hist, lane);
    cnt = vpet::warp_compact_ties(kj, ij, cnt, T, Ti, lane);
    if (lane == 0) atomicAdd(&status[0], 1);
    return key2f(T - 1u);               // the largest float below T
}

constexpr int L1_V = 4;                 // voxels per warp (each loaded draw value serves four)

// Packed fp32 pairs (two lanes of arithmetic per instruction, each rounded as the
// scalar operation would be).
__device__ __forceinline__ unsigned long long pk(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float pk_lo(unsigned long long v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo;
}
__device__ __forceinline__ float pk_hi(unsigned long long v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return hi;
}
// d + w |y - x| on both halves
__device__ __forceinline__ unsigned long long l1_step2(unsigned long long w, unsigned long long y, unsigned long long x,
                                                       unsigned long long d) {
    unsigned long long t, r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(y), "l"(x));
    t &= 0x7FFFFFFF7FFFFFFFull;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(w), "l"(t), "l"(d));
    return r;
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(512, 1) k_l1_scan(const __grid_constant__ L1Args A) {
    extern __shared__ __align__(16) float sm[];
    const int warps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* xbuf = sm;                                        // 2 x [L][L1_TS]: x_l of two tiles' draws
    float* wsh = xbuf + 2 * A.L * L1_TS;                     // [L1_MAXL]: w_l
    float* ys = wsh + L1_MAXL;                               // [warps][L1_V][L1_MAXL]: y_l
    uint32_t* hist = (uint32_t*)(ys + warps * L1_V * L1_MAXL) + wid * 256;
    const int64_t j0 = ((int64_t)blockIdx.x * warps + wid) * L1_V;
    const int seg = blockIdx.y;
    const int64_t tb = (int64_t)seg * A.seg_len;
    const int64_t te = tb + A.seg_len < A.N ? tb + A.seg_len : A.N;
    float* yw = ys + wid * L1_V * L1_MAXL;
    float* kj[L1_V];
    int32_t* ij[L1_V];
    float thr[L1_V];
    int cnt[L1_V];
    bool valid[L1_V];
#pragma unroll
    for (int v = 0; v < L1_V; ++v) {
        const int64_t j = j0 + v;
        valid[v] = j < A.J;
        for (int l = lane; l < A.L; l += 32) yw[v * L1_MAXL + l] = valid[v] ? A.y[j * A.ldy + l] : 0.0f;
        kj[v] = A.keys + ((valid[v] ? j : 0) * A.S + seg) * (int64_t)A.C;
        ij[v] = A.idx + ((valid[v] ? j : 0) * A.S + seg) * (int64_t)A.C;
        thr[v] = __int_as_float(0x7F800000);               // +inf until the first cut
        cnt[v] = 0;
    }
    for (int l = threadIdx.x; l < A.L; l += blockDim.x) wsh[l] = A.w[l];
    const bool any = valid[0];
    // tiles stream through two buffers: the next tile's asynchronous copies are in
    // flight while this one is scanned (draws past the segment are zero-filled)
    auto stage = [&](int64_t t0, float* dst) {
        const int nt = te - t0 < L1_TILE ? (int)(te - t0) : L1_TILE;
        for (int e = threadIdx.x; e < L1_TILE * A.L; e += blockDim.x) {
            const int u = e / A.L, l = e - u * A.L;
            cp_async4(dst + l * L1_TS + u, A.x + (t0 + (u < nt ? u : 0)) * A.ldx + l, u < nt);
        }
        cp_async_commit();
    };
    stage(tb, xbuf);
    int buf = 0;
    for (int64_t t0 = tb; t0 < te; t0 += L1_TILE, buf ^= 1) {
        const int nt = te - t0 < L1_TILE ? (int)(te - t0) : L1_TILE;
        if (t0 + L1_TILE < te) {
            stage(t0 + L1_TILE, xbuf + (buf ^ 1) * A.L * L1_TS);
            cp_async_wait_1();
        } else {
            cp_async_wait_0();
        }
        __syncthreads();                                     // this tile is in shared memory
        const float* xs = xbuf + buf * A.L * L1_TS;
        if (any) {
        // lane draws 2 lane + 64 p + {0, 1} (p < 4), distances in packed pairs
        unsigned long long d2[L1_V][4];
#pragma unroll
        for (int v = 0; v < L1_V; ++v)
#pragma unroll
            for (int q = 0; q < 4; ++q) d2[v][q] = 0ull;
        for (int l = 0; l < A.L; ++l) {                     // frames in order: one fixed summation
            const float wl = wsh[l];
            const unsigned long long w2 = pk(wl, wl);
            unsigned long long x2[4];
            const unsigned long long* xr = (const unsigned long long*)(xs + l * L1_TS) + lane;
#pragma unroll
            for (int q = 0; q < 4; ++q) x2[q] = xr[32 * q];
#pragma unroll
            for (int v = 0; v < L1_V; ++v) {
                const float yl = yw[v * L1_MAXL + l];
                const unsigned long long y2 = pk(yl, yl);
#pragma unroll
                for (int q = 0; q < 4; ++q) d2[v][q] = l1_step2(w2, y2, x2[q], d2[v][q]);
            }
        }
#pragma unroll
        for (int v = 0; v < L1_V; ++v) {
            if (!valid[v]) continue;                         // warp-uniform
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int uu = 64 * (u >> 1) + 2 * lane + (u & 1);
                const float du = (u & 1) ? pk_hi(d2[v][u >> 1]) : pk_lo(d2[v][u >> 1]);
                const bool take = uu < nt && du <= thr[v];
                const uint32_t b = __ballot_sync(0xFFFFFFFFu, take);
                if (take) {
                    const int pos = cnt[v] + __popc(b & ((1u << lane) - 1u));
                    kj[v][pos] = du;
                    ij[v][pos] = (int32_t)(t0 + uu);
                }
                cnt[v] += __popc(b);
            }
            if (cnt[v] > A.C - L1_TILE) {                    // no room for another tile: cut
                __syncwarp();
                thr[v] = cut_list(kj[v], ij[v], cnt[v], A.k, A.C - L1_TILE, hist, lane, A.status);
            }
        }
        }
        __syncthreads();                                     // this buffer is free for the tile after next
    }
#pragma unroll
    for (int v = 0; v < L1_V; ++v)
        if (valid[v] && lane == 0) A.cnt[(j0 + v) * A.S + seg] = cnt[v];
}

// Final k per voxel: exact k-th key, entries at or below it (ties beyond the sort
// buffer by lowest draw index), sorted by (distance, draw index).
__global__ void k_l1_final(const __grid_constant__ L1Args A) {
    extern __shared__ __align__(16) uint8_t fsm[];
    const int warps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* hist = (uint32_t*)fsm + wid * 256;
    unsigned long long* sbuf = (unsigned long long*)(fsm + warps * 1024) + (size_t)wid * A.sortcap;
    const int64_t j = (int64_t)blockIdx.x * warps + wid;
    if (j >= A.J) return;
    float* kj = A.keys + j * A.S * (int64_t)A.C;
    int32_t* ij = A.idx + j * A.S * (int64_t)A.C;
    // the segments' lists, one after another (each moves down: rows of 32 are read
    // before they are written, and every write lands at or below its read)
    int cnt = A.cnt[j * A.S];
    for (int sg = 1; sg < A.S; ++sg) {
        const int c = A.cnt[j * A.S + sg];
        const int src = sg * A.C;
        if (src != cnt)
            for (int b = 0; b < c; b += 32) {
                const int i = b + lane;
                float kv = 0.0f;
                int32_t iv = 0;
                if (i < c) {
                    kv = kj[src + i];
                    iv = ij[src + i];
                }
                __syncwarp();
                if (i < c) {
                    kj[cnt + i] = kv;
                    ij[cnt + i] = iv;
                }
                __syncwarp();
            }
        cnt += c;
    }
    if (cnt > A.k) {
        const uint32_t K = vpet::warp_select(kj, cnt, A.k - 1, 4, hist, lane);
        const vpet::KthKey c = vpet::warp_count_key(kj, cnt, K, lane);
        if (c.n_less + c.n_eq > A.sortcap) {
            const uint32_t Ti = vpet::warp_select_tie_index(kj, ij, cnt, K, A.k - c.n_less - 1, hist, lane);
            cnt = vpet::warp_compact_ties(kj, ij, cnt, K, Ti, lane);
        } else {
            cnt = vpet::warp_compact(kj, ij, cnt, K, A.sortcap, lane);
        }
    }
    int n2 = 32;
    while (n2 < cnt) n2 <<= 1;
    for (int i = lane; i < n2; i += 32)
        sbuf[i] = i < cnt ? (((unsigned long long)f2key(kj[i]) << 32) | (uint32_t)ij[i]) : ~0ull;
    vpet::warp_bitonic_sort(sbuf, n2, lane);
    for (int r = lane; r < A.k; r += 32) {
        const unsigned long long e = r < cnt ? sbuf[r] : ~0ull;
        A.out_idx[j * A.k + r] = r < cnt ? (int32_t)(uint32_t)e : -1;
        A.out_dist[j * A.k + r] = r < cnt ? key2f((uint32_t)(e >> 32)) : __int_as_float(0x7F800000);
    }
}

int l1_capacity(int k) { return (int)vpet_round_up(2 * (int64_t)k + 2 * L1_TILE, 32); }

// Voxels per scan block, and the most draw segments for J voxels: enough blocks for
// two per SM of a 148-SM B300 (at most 16 segments).
constexpr int L1_BLOCK_VOXELS = 16 * L1_V;
int l1_max_segments(int64_t J) {
    const int64_t groups = J > 0 ? vpet_ceil_div(J, L1_BLOCK_VOXELS) : 1;
    const int64_t s = vpet_ceil_div(2 * 148, groups);
    return (int)(s < 1 ? 1 : (s > 16 ? 16 : s));
}
size_t l1_list_bytes(int64_t J, int k) { return (size_t)J * l1_max_segments(J) * (size_t)l1_capacity(k) * 4; }

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" size_t abc_l1_workspace_size(int64_t J, int32_t k) {
    if (J < 0 || k < 1 || k > 2048) return 0;
    return align256(l1_list_bytes(J, k)) * 2 + align256((size_t)J * l1_max_segments(J) * 4) + 512;   // + slack, counter
}

extern "C" int abc_discrepancy_topk_l1(const float* y_dev, int64_t J, int32_t ldy, const float* x_dev, int64_t N,
                                       int32_t ldx, int32_t L, const float* w_host, int32_t k, int32_t* idx_dev,
                                       float* dist_dev, void* workspace_dev, size_t workspace_bytes,
                                       void* stream) {
    vpet::clear_error();
    VPET_ARG(L >= 1 && L <= L1_MAXL, "abc_discrepancy_topk_l1: L must be in 1..%d", L1_MAXL);
    VPET_ARG(k >= 1 && k <= 2048, "abc_discrepancy_topk_l1: k must be in 1..2048");
    VPET_ARG(J >= 0 && J <= 0x7FFFFFFF, "abc_discrepancy_topk_l1: J must be in 0..2^31-1");
    VPET_ARG(N >= k && N <= 0x7FFFFFFF, "abc_discrepancy_topk_l1: need k <= N <= 2^31 - 1");
    VPET_ARG(ldy >= L && ldx >= L, "abc_discrepancy_topk_l1: ldy and ldx must be >= L");
    VPET_ARG(w_host, "abc_discrepancy_topk_l1: null weights");
    L1Args A;
    memset(&A, 0, sizeof A);
    for (int l = 0; l < L; ++l) {
        VPET_ARG(w_host[l] >= 0.0f && w_host[l] < 3.0e38f, "abc_discrepancy_topk_l1: weight %d must be finite, >= 0", l);
        A.w[l] = w_host[l];
    }
    const size_t need = abc_l1_workspace_size(J, k);
    VPET_ARG(workspace_bytes >= need, "abc_discrepancy_topk_l1: workspace %zu < %zu bytes", workspace_bytes, need);
    if (J == 0) return ABC_OK;
    VPET_ARG(y_dev && x_dev && idx_dev && dist_dev && workspace_dev, "abc_discrepancy_topk_l1: null pointer");
    A.y = y_dev;
    A.J = J;
    A.ldy = ldy;
    A.x = x_dev;
    A.N = N;
    A.ldx = ldx;
    A.L = L;
    A.k = k;
    A.C = l1_capacity(k);
    uint8_t* ws = (uint8_t*)(((uintptr_t)workspace_dev + 255) & ~(uintptr_t)255);
    A.keys = (float*)ws;
    A.idx = (int32_t*)(ws + align256(l1_list_bytes(J, k)));
    A.cnt = (int32_t*)(ws + 2 * align256(l1_list_bytes(J, k)));
    // split the draws into segments when there are too few voxel blocks; a segment
    // holds at least four tiles
    int S = l1_max_segments(J);
    const int64_t smax = N / (4 * L1_TILE);
    if (S > smax) S = smax < 1 ? 1 : (int)smax;
    A.seg_len = vpet_round_up(vpet_ceil_div(N, S), L1_TILE);
    A.S = (int)vpet_ceil_div(N, A.seg_len);
    A.out_dist = dist_dev;
    A.out_idx = idx_dev;
    int sortcap = 64;
    while (sortcap < k + 8) sortcap <<= 1;
    A.sortcap = sortcap;
    cudaStream_t s = (cudaStream_t)stream;
    // tie-overflow counter: the last 256 bytes of the workspace
    A.status = (int32_t*)(ws + 2 * align256(l1_list_bytes(J, k)) + align256((size_t)J * l1_max_segments(J) * 4));
    VPET_CUDA(cudaMemsetAsync(A.status, 0, 4, s));
    const int warps = L1_BLOCK_VOXELS / L1_V;
    const size_t smem =
        ((size_t)2 * L * L1_TS + L1_MAXL + (size_t)warps * L1_V * L1_MAXL + (size_t)warps * 256) * 4;
    // kernel attributes are per device: raised once for each device that launches
    static size_t configured[64] = {};
    int dev = 0;
    VPET_CUDA(cudaGetDevice(&dev));
    VPET_ARG(dev >= 0 && dev < 64, "device ordinal %d out of range", dev);
    if (smem > 48 * 1024 && smem > configured[dev]) {
        VPET_CUDA(cudaFuncSetAttribute(k_l1_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured[dev] = smem;
    }
    k_l1_scan<<<dim3((unsigned)vpet_ceil_div(J, (int64_t)L1_BLOCK_VOXELS), (unsigned)A.S), warps * 32, smem, s>>>(A);
    VPET_LAUNCH_CHECK();
    int fw = 8;
    while (fw > 1 && (size_t)fw * (1024 + (size_t)sortcap * 8) > 96 * 1024) fw >>= 1;
    const size_t fsmem = (size_t)fw * (1024 + (size_t)sortcap * 8);
    static size_t fconfigured[64] = {};
    if (fsmem > 48 * 1024 && fsmem > fconfigured[dev]) {
        VPET_CUDA(cudaFuncSetAttribute(k_l1_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
        fconfigured[dev] = fsmem;
    }
    k_l1_final<<<(unsigned)vpet_ceil_div(J, fw), fw * 32, fsmem, s>>>(A);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

extern "C" int abc_l1_status(const void* workspace_dev, int64_t J, int32_t k, int32_t* tie_overflow_host) {
    vpet::clear_error();
    VPET_ARG(workspace_dev && tie_overflow_host && J >= 0 && k >= 1 && k <= 2048, "abc_l1_status: bad argument");
    const uint8_t* ws = (const uint8_t*)(((uintptr_t)workspace_dev + 255) & ~(uintptr_t)255);
    const int32_t* st =
        (const int32_t*)(ws + 2 * align256(l1_list_bytes(J, k)) + align256((size_t)J * l1_max_segments(J) * 4));
    VPET_CUDA(cudaMemcpy(tie_overflow_host, st, 4, cudaMemcpyDeviceToHost));
    return ABC_OK;
}
