// Reliability check of the learned path and its calibration (the learned proposal is a
// workload extension with no counterpart in the paper): which voxels fall back to the global
// path (Algorithm 1), the gather of their rows and the scatter of the global results, and
// the quantile of the global path's relative median accepted distance that sets the
// threshold of the check.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace {

constexpr int FB_BLOCK = 1024;

// The fallback predicate, the same in the counting and the writing pass.
__device__ __forceinline__ bool falls_back(const float* ess, const float* dmed, const float* ynorm, int64_t j,
                                           float ess_min, float rel_max) {
    const float e = ess[j];
    if (!(e >= ess_min)) return true;                  // a NaN ESS counts as unreliable
    return rel_max > 0.0f && dmed[j] > rel_max * ynorm[j];
}

__global__ void __launch_bounds__(FB_BLOCK) k_fb_count(const float* __restrict__ ess, const float* __restrict__ dmed,
                                                       const float* __restrict__ ynorm, int64_t J, float ess_min,
                                                       float rel_max, int32_t* __restrict__ cnt) {
    const int64_t j = (int64_t)blockIdx.x * FB_BLOCK + threadIdx.x;
    const bool f = j < J && falls_back(ess, dmed, ynorm, j, ess_min, rel_max);
    const int c = __syncthreads_count(f);
    if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

// Exclusive scan of the nb block counts (one block); the total goes to *total.
__global__ void __launch_bounds__(FB_BLOCK) k_fb_scan(const int32_t* __restrict__ cnt, int64_t nb,
                                                      int32_t* __restrict__ off, int32_t* __restrict__ total) {
    __shared__ int32_t wsum[FB_BLOCK / 32];
    __shared__ int32_t carry;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += FB_BLOCK) {
        const int64_t b = b0 + threadIdx.x;
        const int32_t v = b < nb ? cnt[b] : 0;
        int32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[wp] = incl;
        __syncthreads();
        if (wp == 0) {
            int32_t s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t u = __shfl_up_sync(0xFFFFFFFFu, s, o);
                if (lane >= o) s += u;
            }
            wsum[lane] = s;                              // inclusive over warps
        }
        __syncthreads();
        const int32_t before = carry + (wp > 0 ? wsum[wp - 1] : 0) + incl - v;
        if (b < nb) off[b] = before;
        __syncthreads();
        if (threadIdx.x == FB_BLOCK - 1) carry += wsum[FB_BLOCK / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// Rows of the fallback voxels, ascending: the block's offset plus the voxel's rank in it.
__global__ void __launch_bounds__(FB_BLOCK) k_fb_write(const float* __restrict__ ess, const float* __restrict__ dmed,
                                                       const float* __restrict__ ynorm, int64_t J, float ess_min,
                                                       float rel_max, const int32_t* __restrict__ off,
                                                       int32_t* __restrict__ rows) {
    __shared__ int32_t wcnt[FB_BLOCK / 32];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * FB_BLOCK + threadIdx.x;
    const bool f = j < J && falls_back(ess, dmed, ynorm, j, ess_min, rel_max);
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, f);
    if (lane == 0) wcnt[wp] = __popc(bal);
    __syncthreads();
    int32_t pos = off[blockIdx.x];
    for (int q = 0; q < wp; ++q) pos += wcnt[q];
    pos += __popc(bal & ((1u << lane) - 1u));
    if (f) rows[pos] = (int32_t)j;
}

// One warp per listed row (i < *count): dst row i <- src row rows[i], or (scatter) dst row
// rows[i] <- src row i.
template <bool SCATTER>
__global__ void k_move_rows(const float* __restrict__ src, int32_t ld_src, const int32_t* __restrict__ rows,
                            const int32_t* __restrict__ count, int64_t max_rows, int32_t width, float* __restrict__ dst,
                            int32_t ld_dst) {
    const int lane = threadIdx.x & 31;
    const int64_t n = *count < max_rows ? *count : max_rows;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
         i += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const int64_t r = rows[i];
        const float* s = SCATTER ? src + i * ld_src : src + r * ld_src;
        float* d = SCATTER ? dst + r * ld_dst : dst + i * ld_dst;
        for (int c = lane; c < width; c += 32) d[c] = s[c];
    }
}

// ------------------------------------------------------------------ quantile
// Order-preserving image of a float in uint32 (NaN above +inf).
__device__ __forceinline__ uint32_t qkey(float f) {
    if (f != f) return 0xFFFFFFFFu;
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// keys[j] = image of dist[j k + col] / (sum_l w_l y_jl^2), one thread per voxel
struct QW {
    float w[64];
};
__global__ void k_q_keys(const float* __restrict__ dist, int64_t J, int32_t k, int32_t col, const float* __restrict__ y,
                         int32_t ldy, int32_t L, QW W, uint32_t* __restrict__ keys) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    const float* yr = y + j * ldy;
    float yn = 0.0f;
    for (int l = 0; l < L; ++l) yn = fmaf(W.w[l] * yr[l], yr[l], yn);
    keys[j] = qkey(dist[j * k + col] / yn);
}

// Radix selection state of two ranks: prefix and mask of the digits fixed so far, the rank
// left within them, then two 256-bin histograms.
struct QState {
    uint32_t prefix[2];
    uint32_t mask;
    uint32_t rank[2];
    uint32_t pad[3];
    uint32_t hist[2][256];
};

__global__ void k_q_hist(const uint32_t* __restrict__ keys, int64_t J, int shift, QState* __restrict__ S) {
    __shared__ uint32_t h[2][256];
    for (int i = threadIdx.x; i < 512; i += blockDim.x) h[i >> 8][i & 255] = 0;
    __syncthreads();
    const uint32_t mask = S->mask, p0 = S->prefix[0], p1 = S->prefix[1];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < J; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = keys[j];
        const uint32_t d = (key >> shift) & 0xFFu;
        if ((key & mask) == p0) atomicAdd(&h[0][d], 1u);
        if ((key & mask) == p1) atomicAdd(&h[1][d], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 512; i += blockDim.x)
        if (h[i >> 8][i & 255]) atomicAdd(&S->hist[i >> 8][i & 255], h[i >> 8][i & 255]);
}

// one thread per rank: the digit whose bin holds the rank; histograms cleared for the next digit
__global__ void k_q_pick(int shift, QState* __restrict__ S) {
    const int s = threadIdx.x;
    if (s < 2) {
        uint32_t cum = 0, r = S->rank[s];
        int b = 0;
        for (; b < 255; ++b) {
            if (r < cum + S->hist[s][b]) break;
            cum += S->hist[s][b];
        }
        S->prefix[s] |= (uint32_t)b << shift;
        S->rank[s] = r - cum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 512; i += blockDim.x) S->hist[i >> 8][i & 255] = 0;
    if (threadIdx.x == 0) S->mask |= 0xFFu << shift;
}

float key_to_float(uint32_t k) {
    if (k == 0xFFFFFFFFu) return NAN;
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

int64_t fb_blocks(int64_t J) { return (J + FB_BLOCK - 1) / FB_BLOCK; }

}  // namespace

extern "C" size_t abc_fallback_scratch_size(int64_t J) {
    if (J < 1 || J > INT32_MAX) return 0;
    return (size_t)(2 * fb_blocks(J)) * sizeof(int32_t) + 256;
}

extern "C" int abc_fallback_rows(const float* ess_dev, const float* dmed_dev, const float* ynorm_dev, int64_t J,
                                 int32_t k, float rel_max, int32_t* rows_dev, int32_t* count_dev, void* scratch_dev,
                                 size_t scratch_bytes, void* stream) {
    vpet::clear_error();
    VPET_ARG(J >= 1 && J <= INT32_MAX, "abc_fallback_rows: J must be in 1 .. 2^31 - 1");
    VPET_ARG(k >= 1, "abc_fallback_rows: k must be positive");
    VPET_ARG(ess_dev && rows_dev && count_dev && scratch_dev, "abc_fallback_rows: null pointer");
    VPET_ARG(!(rel_max > 0.0f) || (dmed_dev && ynorm_dev), "abc_fallback_rows: rel_max > 0 needs dmed and ynorm");
    VPET_ARG(scratch_bytes >= abc_fallback_scratch_size(J), "abc_fallback_rows: scratch needs %zu bytes (got %zu)",
             abc_fallback_scratch_size(J), scratch_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nb = fb_blocks(J);
    int32_t* cnt = (int32_t*)scratch_dev;
    int32_t* off = cnt + nb;
    const float ess_min = (float)k / 4.0f;
    const float rm = rel_max > 0.0f ? rel_max : 0.0f;
    k_fb_count<<<(unsigned)nb, FB_BLOCK, 0, s>>>(ess_dev, dmed_dev, ynorm_dev, J, ess_min, rm, cnt);
    VPET_LAUNCH_CHECK();
    k_fb_scan<<<1, FB_BLOCK, 0, s>>>(cnt, nb, off, count_dev);
    VPET_LAUNCH_CHECK();
    k_fb_write<<<(unsigned)nb, FB_BLOCK, 0, s>>>(ess_dev, dmed_dev, ynorm_dev, J, ess_min, rm, off, rows_dev);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

static int move_rows(bool scatter, const float* src_dev, int32_t ld_src, const int32_t* rows_dev,
                     const int32_t* count_dev, int64_t max_rows, int32_t width, float* dst_dev, int32_t ld_dst,
                     void* stream) {
    VPET_ARG(src_dev && rows_dev && count_dev && dst_dev, "abc_gather_rows / abc_scatter_rows: null pointer");
    VPET_ARG(max_rows >= 0 && width >= 1 && ld_src >= width && ld_dst >= width,
             "abc_gather_rows / abc_scatter_rows: bad sizes (width %d, ld_src %d, ld_dst %d)", width, ld_src, ld_dst);
    if (max_rows == 0) return ABC_OK;
    int dev = 0, sms = 0;
    VPET_CUDA(cudaGetDevice(&dev));
    VPET_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t want = (max_rows + 7) / 8;
    const unsigned grid = (unsigned)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    cudaStream_t s = (cudaStream_t)stream;
    if (scatter)
        k_move_rows<true><<<grid, 256, 0, s>>>(src_dev, ld_src, rows_dev, count_dev, max_rows, width, dst_dev, ld_dst);
    else
        k_move_rows<false><<<grid, 256, 0, s>>>(src_dev, ld_src, rows_dev, count_dev, max_rows, width, dst_dev, ld_dst);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

extern "C" int abc_gather_rows(const float* src_dev, int32_t ld_src, const int32_t* rows_dev, const int32_t* count_dev,
                               int64_t max_rows, int32_t width, float* dst_dev, int32_t ld_dst, void* stream) {
    vpet::clear_error();
    return move_rows(false, src_dev, ld_src, rows_dev, count_dev, max_rows, width, dst_dev, ld_dst, stream);
}

extern "C" int abc_scatter_rows(const float* src_dev, int32_t ld_src, const int32_t* rows_dev, const int32_t* count_dev,
                                int64_t max_rows, int32_t width, float* dst_dev, int32_t ld_dst, void* stream) {
    vpet::clear_error();
    return move_rows(true, src_dev, ld_src, rows_dev, count_dev, max_rows, width, dst_dev, ld_dst, stream);
}

extern "C" size_t abc_quantile_scratch_size(int64_t J) {
    if (J < 1 || J > INT32_MAX) return 0;
    return (size_t)J * sizeof(uint32_t) + 256 + sizeof(QState);
}

extern "C" int abc_median_rel_quantile(const float* dist_dev, int64_t J, int32_t k, const float* y_dev, int32_t ldy,
                                       int32_t L, const float* w_host, double q, float* out_host, void* scratch_dev,
                                       size_t scratch_bytes, void* stream) {
    vpet::clear_error();
    VPET_ARG(J >= 1 && J <= INT32_MAX, "abc_median_rel_quantile: J must be in 1 .. 2^31 - 1");
    VPET_ARG(k >= 1 && L >= 1 && L <= 64 && ldy >= L, "abc_median_rel_quantile: bad k, L or ldy");
    VPET_ARG(q >= 0.0 && q <= 1.0, "abc_median_rel_quantile: q must be in [0, 1]");
    VPET_ARG(dist_dev && y_dev && w_host && out_host && scratch_dev, "abc_median_rel_quantile: null pointer");
    VPET_ARG(scratch_bytes >= abc_quantile_scratch_size(J), "abc_median_rel_quantile: scratch needs %zu bytes (got %zu)",
             abc_quantile_scratch_size(J), scratch_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    QW W;
    memset(&W, 0, sizeof W);
    for (int l = 0; l < L; ++l) W.w[l] = w_host[l];
    uint32_t* keys = (uint32_t*)scratch_dev;
    QState* S = (QState*)(((uintptr_t)(keys + J) + 255) & ~(uintptr_t)255);
    // ranks of numpy's linear interpolation: h = q (J - 1), order statistics floor(h) and the next
    const double h = q * (double)(J - 1);
    const int64_t r0 = (int64_t)floor(h), r1 = r0 + 1 < J ? r0 + 1 : r0;
    QState init;
    memset(&init, 0, sizeof init);
    init.rank[0] = (uint32_t)r0;
    init.rank[1] = (uint32_t)r1;
    VPET_CUDA(cudaMemcpyAsync(S, &init, sizeof init, cudaMemcpyHostToDevice, s));
    k_q_keys<<<(unsigned)((J + 255) / 256), 256, 0, s>>>(dist_dev, J, k, (k - 1) / 2, y_dev, ldy, L, W, keys);
    VPET_LAUNCH_CHECK();
    int dev = 0, sms = 0;
    VPET_CUDA(cudaGetDevice(&dev));
    VPET_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t want = (J + 255) / 256;
    const unsigned grid = (unsigned)(want < (int64_t)sms * 4 ? want : (int64_t)sms * 4);
    for (int shift = 24; shift >= 0; shift -= 8) {
        k_q_hist<<<grid, 256, 0, s>>>(keys, J, shift, S);
        VPET_LAUNCH_CHECK();
        k_q_pick<<<1, 256, 0, s>>>(shift, S);
        VPET_LAUNCH_CHECK();
    }
    uint32_t pre[2];
    VPET_CUDA(cudaMemcpyAsync(pre, S->prefix, sizeof pre, cudaMemcpyDeviceToHost, s));
    VPET_CUDA(cudaStreamSynchronize(s));
    const double a = key_to_float(pre[0]), b = key_to_float(pre[1]), t = h - (double)r0;
    // numpy's lerp: a + t (b - a), or b - (1 - t) (b - a) from the upper end
    const double d = b - a;
    *out_host = (float)(t >= 0.5 ? b - d * (1.0 - t) : a + d * t);
    return ABC_OK;
}
