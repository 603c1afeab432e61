// Posterior model probabilities and posterior summaries over each voxel's
// accepted draws (Sec. II-B Eq. 6, Sec. II-D, Sec. III-B).  One warp per voxel;
// compensated fp32 sums for means and variances; credible intervals from exact
// order statistics (radix selection, type-7 interpolation).
#include <string.h>

#include "common.cuh"

namespace {

constexpr int MAXM = 16;

struct Segs {
    int M;
    int64_t off[MAXM + 1];
};

__device__ __forceinline__ int model_of(int64_t i, const Segs& s) {
    int m = 0;
    while (m < s.M && i >= s.off[m + 1]) ++m;
    return (i >= s.off[0] && m < s.M) ? m : -1;
}

__global__ void k_model_select(const int32_t* __restrict__ idx, int64_t J, int k, Segs S, float* __restrict__ prob,
                               int8_t* __restrict__ pref) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= J) return;
    int cnt[MAXM];
#pragma unroll
    for (int m = 0; m < MAXM; ++m) cnt[m] = 0;
    // four 32-index chunks per round, their loads in flight together
    for (int base = 0; base < k; base += 128) {
        int32_t id[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = base + 32 * u + lane;
            id[u] = r < k ? idx[j * k + r] : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int m = base + 32 * u + lane < k ? model_of(id[u], S) : -1;
#pragma unroll
            for (int q = 0; q < MAXM; ++q) cnt[q] += (q == m);
        }
    }
    int best = 0, bestc = -1;
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
        int c = cnt[m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if (m < S.M) {
            if (lane == 0) prob[j * S.M + m] = (float)c / (float)k;
            if (c > bestc) { bestc = c; best = m; }
        }
    }
    if (lane == 0) pref[j] = (int8_t)best;
}

struct SumParams {
    Segs S;
    int nparams[MAXM];
    int has_ki[MAXM];
    int ki[3];
    int Pmax, ncols, k, p2, ldt;
};

// Compensated fp32 accumulation (Neumaier's variant of Kahan summation): the
// running sum s and the lost low-order parts c; the value is s + c.
struct CSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float t = s + v;
        c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
        s = t;
    }
};

// Warp total of per-lane compensated sums: pairs of (sum, compensation) are
// combined the same way along a butterfly, so every lane gets the same value.
__device__ __forceinline__ float warp_csum(CSum a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xFFFFFFFFu, a.s, o), c2 = __shfl_xor_sync(0xFFFFFFFFu, a.c, o);
        a.c += c2;
        a.add(s2);
    }
    return a.s + a.c;
}

__device__ __forceinline__ uint32_t f2o(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float o2f(uint32_t k) { return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k); }

// The r-th smallest (0-based) of the n floats in s (shared memory), exactly: a
// 4-level radix select on the order-preserving integer image, 8 bits per level
// (lanes with the same digit add their count once); hist is 256 words of this
// warp's shared memory.
__device__ float warp_kth_radix(const float* s, int n, int r, uint32_t* hist, int lane) {
    uint32_t prefix = 0;
    for (int lv = 0; lv < 4; ++lv) {
        const int shift = 24 - 8 * lv;
        const uint32_t mask = lv == 0 ? 0u : (0xFFFFFFFFu << (shift + 8));
        for (int b = lane; b < 256; b += 32) hist[b] = 0;
        __syncwarp();
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            const uint32_t k = i < n ? f2o(s[i]) : 0u;
            const uint32_t bin = (i < n && (k & mask) == prefix) ? (k >> shift) & 255u : (0x100u | (uint32_t)lane);
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, bin);
            if (bin < 256u && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
        }
        __syncwarp();
        uint32_t loc[8], sum = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) { loc[b] = hist[lane * 8 + b]; sum += loc[b]; }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += v;
        }
        uint32_t c = incl - sum;
        int found = -1, nr = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            if (found < 0 && c + loc[b] > (uint32_t)r) { found = lane * 8 + b; nr = r - (int)c; }
            c += loc[b];
        }
        const uint32_t who = __ballot_sync(0xFFFFFFFFu, found >= 0);
        const int src = __ffs(who) - 1;
        const int bin = __shfl_sync(0xFFFFFFFFu, found, src);
        r = __shfl_sync(0xFFFFFFFFu, nr, src);
        prefix |= (uint32_t)bin << shift;
        __syncwarp();
    }
    return o2f(prefix);
}

// Order statistics of ranks rk[0] <= rk[1] and rk[2] <= rk[3] (each in [0, n)) of
// 32 < n <= 256 floats in s, exactly, for ranks near the two ends (the 95 % interval's):
// each lane sorts the order-preserving integer images of its values s[lane + 32 i] (at
// most 8) in registers; the warp then takes values in ascending order from the low end,
// rk[1] + 1 rounds, and in descending order from the high end, n - rk[2] rounds, both ends
// in the same loop, one value per end and round (the smallest, resp. largest, of the lanes'
// next values by one warp reduction; on equal values the lowest lane's), so the value taken
// in round r is the order statistic of that rank, duplicates included.
__device__ __forceinline__ void warp_tails4(const float* s, int n, const int (&rk)[4], int lane, float (&out)[4]) {
    uint32_t v[8];
    int c = 0;                                     // values this lane holds
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = lane + 32 * i;
        v[i] = idx < n ? f2o(s[idx]) : 0xFFFFFFFFu;
        c += idx < n;
    }
    // odd-even transposition sort: eight phases order eight keys (the pads last)
#pragma unroll
    for (int ph = 0; ph < 8; ++ph)
#pragma unroll
        for (int i = ph & 1; i + 1 < 8; i += 2) {
            const uint32_t a = min(v[i], v[i + 1]), b = max(v[i], v[i + 1]);
            v[i] = a;
            v[i + 1] = b;
        }
    auto pick = [&](int i) {
        uint32_t h = v[0];
#pragma unroll
        for (int q = 1; q < 8; ++q) h = i == q ? v[q] : h;
        return h;
    };
    const int rl = rk[1] + 1, ru = n - rk[2];     // rounds at the low and the high end
    const int rounds = rl > ru ? rl : ru;
    int lo = 0, hi = c - 1;
    uint32_t hl = c > 0 ? v[0] : 0xFFFFFFFFu, hh = c > 0 ? pick(hi) : 0u;
    uint32_t o[4] = {0u, 0u, 0u, 0u};
    for (int r = 0; r < rounds; ++r) {
        const uint32_t ml = __reduce_min_sync(0xFFFFFFFFu, hl);
        const uint32_t mh = __reduce_max_sync(0xFFFFFFFFu, hh);
        if (r < rl) {
            const uint32_t who = __ballot_sync(0xFFFFFFFFu, lo < c && hl == ml);
            if (lane == __ffs(who) - 1) {
                ++lo;
                hl = lo < c ? pick(lo) : 0xFFFFFFFFu;
            }
            if (r == rk[0]) o[0] = ml;
            if (r == rk[1]) o[1] = ml;
        }
        if (r < ru) {
            const uint32_t who = __ballot_sync(0xFFFFFFFFu, hi >= 0 && hh == mh);
            if (lane == __ffs(who) - 1) {
                --hi;
                hh = hi >= 0 ? pick(hi) : 0u;
            }
            if (n - 1 - r == rk[3]) o[3] = mh;
            if (n - 1 - r == rk[2]) o[2] = mh;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = o2f(o[q]);
}

// Order statistics of ranks rk[0..3] (each in [0, n)) of the n floats in s,
// exactly, with one histogram: 256 equal-width bins over [min, max] locate the
// bin of each rank; the members of those bins (at most 256 in all) are gathered
// into hist and each rank resolved by counting within its bin.  Crowded bins
// (or an unbounded range) take the radix select per rank.
// mn / mx: this lane's minimum and maximum over its values s[lane + 32 i].
__device__ void warp_order4(const float* s, int n, const int (&rk)[4], uint32_t* hist, int lane, float mn, float mx,
                            float (&out)[4]) {
    if (n <= 32) {
        // one value per lane: a bitonic sort across the warp's registers
        float x = lane < n ? s[lane] : __int_as_float(0x7F800000);
#pragma unroll
        for (int size = 2; size <= 32; size <<= 1)
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                const float y = __shfl_xor_sync(0xFFFFFFFFu, x, stride);
                const bool keep_min = ((lane & stride) == 0) == ((lane & size) == 0 || size == 32);
                x = keep_min ? fminf(x, y) : fmaxf(x, y);
            }
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] = __shfl_sync(0xFFFFFFFFu, x, rk[q]);
        return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    }
    if (mn == mx) {
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] = mn;
        return;
    }
    const float span = mx - mn;
    if (!(span < 3.0e38f)) {
        for (int q = 0; q < 4; ++q) out[q] = warp_kth_radix(s, n, rk[q], hist, lane);
        return;
    }
    const float scale = 256.0f / span;
    auto bin_of = [&](float v) -> int {
        const float t = (v - mn) * scale;
        return t < 255.0f ? (int)t : 255;
    };
    for (int b = lane; b < 256; b += 32) hist[b] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) atomicAdd(&hist[bin_of(s[i])], 1u);
    __syncwarp();
    uint32_t loc[8], sum = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) { loc[b] = hist[lane * 8 + b]; sum += loc[b]; }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t excl = incl - sum;
    int tb[4], tbelow[4], tcnt[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t c = excl;
        int found = -1, below = 0, inbin = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            if (found < 0 && c + loc[b] > (uint32_t)rk[q]) { found = lane * 8 + b; below = (int)c; inbin = (int)loc[b]; }
            c += loc[b];
        }
        const uint32_t who = __ballot_sync(0xFFFFFFFFu, found >= 0);
        const int src = __ffs(who) - 1;
        tb[q] = __shfl_sync(0xFFFFFFFFu, found, src);
        tbelow[q] = __shfl_sync(0xFFFFFFFFu, below, src);
        tcnt[q] = __shfl_sync(0xFFFFFFFFu, inbin, src);
    }
    __syncwarp();   // the histogram is in registers now; its words become the gather buffer
    float* buf = (float*)hist;
    int m = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        float v = 0.0f;
        bool in = false;
        if (i < n) {
            v = s[i];
            const int b = bin_of(v);
            in = b == tb[0] || b == tb[1] || b == tb[2] || b == tb[3];
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, in);
        const int pos = m + __popc(bal & ((1u << lane) - 1u));
        if (in && pos < 256) buf[pos] = v;
        m += __popc(bal);
    }
    __syncwarp();
    if (m > 256) {
        for (int q = 0; q < 4; ++q) out[q] = warp_kth_radix(s, n, rk[q], hist, lane);
        return;
    }
    if (m > 64) {
        // many members (typically many equal values): sort them; the members of the
        // target bins then follow one another in bin order, so rank r of bin b sits at
        // (members of the lower target bins) + (r - keys below bin b)
        int m2 = 64;
        while (m2 < m) m2 <<= 1;
        for (int i = m + lane; i < m2; i += 32) buf[i] = __int_as_float(0x7F800000);
        for (int size = 2; size <= m2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                __syncwarp();
                for (int t = lane; t < (m2 >> 1); t += 32) {
                    const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                    const float a = buf[lo], b = buf[hi];
                    if ((a > b) == ((lo & size) == 0)) {
                        buf[lo] = b;
                        buf[hi] = a;
                    }
                }
            }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int off = 0;
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) {
                bool first = tb[q2] < tb[q];
#pragma unroll
                for (int q3 = 0; q3 < q2; ++q3) first = first && tb[q3] != tb[q2];
                if (first) off += tcnt[q2];
            }
            out[q] = buf[off + rk[q] - tbelow[q]];
        }
        __syncwarp();
        return;
    }
    float res[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    uint32_t got = 0;
    for (int a = lane; a < m; a += 32) {
        const float v = buf[a];
        const int bv = bin_of(v);
        int lt = 0, eq = 0;
        for (int u = 0; u < m; ++u) {
            const float w = buf[u];
            if (bin_of(w) == bv) {
                lt += w < v;
                eq += w == v;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (tb[q] == bv && tbelow[q] + lt <= rk[q] && rk[q] < tbelow[q] + lt + eq) { res[q] = v; got |= 1u << q; }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t who = __ballot_sync(0xFFFFFFFFu, (got >> q) & 1u);
        out[q] = __shfl_sync(0xFFFFFFFFu, res[q], who ? __ffs(who) - 1 : 0);
    }
    __syncwarp();
}


// ROWS (at most 8 parameters, and the warp's rows fit): each accepted draw's parameter row is
// read once, with 16-byte loads where rows are 16-byte aligned (vec4), into the warp's
// column-major table R (ncols columns of p2 floats, K_i computed as the row arrives), and the
// column statistics read R; otherwise each column is gathered through the selected draw
// indices into one column buffer.  The sums visit the values in the same order either way.
template <bool ROWS>
__global__ void k_summarize(const float* __restrict__ theta, const int32_t* __restrict__ idx, int64_t J,
                            const int8_t* __restrict__ pref, SumParams Q, float* __restrict__ mean,
                            float* __restrict__ sd, float* __restrict__ lo, float* __restrict__ hi, bool vec4) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int warps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t* sel = (int32_t*)sm + (size_t)wid * Q.p2;
    float* vals = (float*)(sm + (size_t)warps * Q.p2 * 4) + (size_t)wid * Q.p2;
    uint32_t* hist = (uint32_t*)(sm + (size_t)warps * Q.p2 * 8) + (size_t)wid * 256;
    float* R = (float*)sm + (size_t)wid * Q.ncols * Q.p2;
    if (ROWS) hist = (uint32_t*)(sm + (size_t)warps * Q.ncols * Q.p2 * 4) + (size_t)wid * 256;
    const int64_t j = (int64_t)blockIdx.x * warps + wid;
    if (j >= J) return;
    const int pm = pref ? (int)pref[j] : -1;
    int P = pm >= 0 ? Q.nparams[pm] : Q.Pmax;
    int ki = pm >= 0 ? Q.has_ki[pm] : 1;
    if (pm < 0)
        for (int m = 0; m < Q.S.M; ++m) {
            if (Q.nparams[m] < P) P = Q.nparams[m];
            if (!Q.has_ki[m]) ki = 0;
        }
    // accepted draws of the summarised model, in accepted order
    int n = 0;
    for (int base = 0; base < Q.k; base += 128) {
        int32_t id[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = base + 32 * u + lane;
            id[u] = r < Q.k ? idx[j * Q.k + r] : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool take = id[u] >= 0 && (pm < 0 || model_of(id[u], Q.S) == pm);
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, take);
            const int pos = n + __popc(b & ((1u << lane) - 1u));
            if (ROWS) {
                if (take) {
                    const float* th = theta + (int64_t)id[u] * Q.ldt;
                    float r8[8];
                    if (vec4) {
                        const float4 a = __ldg((const float4*)th);
                        const float4 c = Q.Pmax > 4 ? __ldg((const float4*)th + 1) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        r8[0] = a.x; r8[1] = a.y; r8[2] = a.z; r8[3] = a.w;
                        r8[4] = c.x; r8[5] = c.y; r8[6] = c.z; r8[7] = c.w;
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q) r8[q] = q < Q.Pmax ? th[q] : 0.0f;
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (q < Q.Pmax) R[(size_t)q * Q.p2 + pos] = r8[q];
                    if (ki) {
                        const float K1 = th[Q.ki[0]], k2 = th[Q.ki[1]], k3 = th[Q.ki[2]];
                        R[(size_t)Q.Pmax * Q.p2 + pos] = K1 * k3 / (k2 + k3);
                    }
                }
            } else if (take) {
                sel[pos] = id[u];
            }
            n += __popc(b);
        }
    }
    __syncwarp();
    const float qnan = __int_as_float(0x7FC00000);
    // type-7 quantiles from the two order statistics around each level; the position
    // h = (n - 1) q is formed in fp64 (exact floor at integer h), once per voxel: it
    // depends on n alone, and fp64 issues slowly here
    int rk[4];
    float fr[2];
    {
        const double qs[2] = {0.025, 0.975};
        for (int t = 0; t < 2; ++t) {
            const double h = (n - 1) * qs[t];
            const int a = (int)floor(h);
            fr[t] = (float)(h - a);
            rk[2 * t] = a;
            rk[2 * t + 1] = a + 1 < n ? a + 1 : n - 1;
        }
    }
    for (int col = 0; col < Q.ncols; ++col) {
        const bool isk = col == Q.Pmax;
        float o0 = qnan, o1 = qnan, o2 = qnan, o3 = qnan;
        if (n > 0 && ((isk && ki) || (!isk && col < P))) {
            // fp32 throughout (compensated sums): the values are fp32 and the sums'
            // relative error stays near 2^-24 for any k
            // eight 32-value rounds per gather, their loads in flight together
            const float* cv = ROWS ? R + (size_t)col * Q.p2 : vals;   // the column's values
            CSum s;
            float mn = 3.0e38f, mx = -3.0e38f;
            for (int i0 = 0; i0 < n; i0 += 256) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + 32 * u + lane;
                    v[u] = 0.0f;
                    if (ROWS) {
                        if (i < n) v[u] = cv[i];
                    } else if (i < n) {
                        const float* th = theta + (int64_t)sel[i] * Q.ldt;
                        if (isk) {
                            const float K1 = th[Q.ki[0]], k2 = th[Q.ki[1]], k3 = th[Q.ki[2]];
                            v[u] = K1 * k3 / (k2 + k3);
                        } else {
                            v[u] = th[col];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + 32 * u + lane;
                    if (i < n) {
                        if (!ROWS) vals[i] = v[u];
                        s.add(v[u]);
                        mn = fminf(mn, v[u]);
                        mx = fmaxf(mx, v[u]);
                    }
                }
            }
            const float mu = warp_csum(s) / (float)n;
            CSum ss;
            __syncwarp();
            for (int i = lane; i < n; i += 32) {
                const float e = cv[i] - mu;
                ss.add(e * e);
            }
            const float sst = warp_csum(ss);
            float qv[2], os[4];
            if (n > 32 && n <= 256) warp_tails4(cv, n, rk, lane, os);
            else warp_order4(cv, n, rk, hist, lane, mn, mx, os);
            for (int t = 0; t < 2; ++t) qv[t] = fmaf(fr[t], os[2 * t + 1] - os[2 * t], os[2 * t]);
            o0 = mu;
            o1 = n > 1 ? sqrtf(sst / (float)(n - 1)) : 0.0f;
            o2 = qv[0];
            o3 = qv[1];
            __syncwarp();
        }
        if (lane == 0) {
            mean[j * Q.ncols + col] = o0;
            sd[j * Q.ncols + col] = o1;
            lo[j * Q.ncols + col] = o2;
            hi[j * Q.ncols + col] = o3;
        }
    }
}

// ---------------------------------------------------------------- response band
// lp-ntPET response function k2a(t) / k2a = 1 + (gamma / k2a) g(t) (Sec. II-D), g
// the gamma variate normalised to 1 at t_P: g = 0 before t_D, x^alpha e^{alpha (1 - x)}
// with x = (t - t_D) / (t_P - t_D) after.
constexpr int RESP_MAXT = 256;

struct RespParams {
    int64_t first, last;      // the lp-ntPET draws: global indices [first, last)
    int ldt, k, T, p2;
    float t[RESP_MAXT];
};

__device__ __forceinline__ float gamma_variate_at(float t, float tD, float tPmD, float alpha) {
    if (t < tD) return 0.0f;
    const float x = (t - tD) / tPmD;
    if (alpha == 0.0f) return 1.0f;
    if (x == 0.0f) return 0.0f;
    return expf(alpha * (logf(x) + 1.0f - x));
}

// One warp per voxel: the accepted lp-ntPET draws' (gamma / k2a, t_D, t_P - t_D,
// alpha) go to this warp's shared memory once; then per time the responses, their
// compensated mean and the two type-7 quantiles (four order statistics, one histogram).
__global__ void k_response_cri(const float* __restrict__ theta, const int32_t* __restrict__ idx, int64_t J,
                               const __grid_constant__ RespParams Q, float* __restrict__ mean,
                               float* __restrict__ lo, float* __restrict__ hi) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int warps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* cg = (float*)sm + (size_t)wid * 5 * Q.p2;
    float* td = cg + Q.p2;
    float* tw = td + Q.p2;
    float* al = tw + Q.p2;
    float* vals = al + Q.p2;
    uint32_t* hist = (uint32_t*)((float*)sm + (size_t)warps * 5 * Q.p2) + (size_t)wid * 256;
    const int64_t j = (int64_t)blockIdx.x * warps + wid;
    if (j >= J) return;
    int n = 0;
    for (int base = 0; base < Q.k; base += 128) {
        int32_t id[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = base + 32 * u + lane;
            id[u] = r < Q.k ? idx[j * Q.k + r] : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool take = base + 32 * u + lane < Q.k && (int64_t)id[u] >= Q.first && (int64_t)id[u] < Q.last;
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, take);
            if (take) {
                const int pos = n + __popc(b & ((1u << lane) - 1u));
                const float* th = theta + (int64_t)id[u] * Q.ldt;
                const float k2a = th[1] / (1.0f + th[2]);
                cg[pos] = th[3] / k2a;
                td[pos] = th[4];
                tw[pos] = th[5];
                al[pos] = th[6];
            }
            n += __popc(b);
        }
    }
    __syncwarp();
    const float qnan = __int_as_float(0x7FC00000);
    int rk[4];
    float fr[2];
    const double qs[2] = {0.025, 0.975};
    for (int q = 0; q < 2; ++q) {
        const double h = (n - 1) * qs[q];
        const int a = (int)floor(h);
        fr[q] = (float)(h - a);
        rk[2 * q] = a;
        rk[2 * q + 1] = a + 1 < n ? a + 1 : n - 1;
    }
    for (int m = 0; m < Q.T; ++m) {
        float o0 = qnan, o1 = qnan, o2 = qnan;
        if (n > 0) {
            // responses equal to 1 (before t_D, gamma = 0) are only counted; the others are
            // compacted into vals, and a rank falls on 1, below the ones or above them
            const float t = Q.t[m];
            CSum s;
            float mn = 3.0e38f, mx = -3.0e38f;
            int nb = 0, nv = 0;
            for (int i0 = 0; i0 < n; i0 += 32) {
                const int i = i0 + lane;
                float v = 1.0f;
                if (i < n) v = 1.0f + cg[i] * gamma_variate_at(t, td[i], tw[i], al[i]);
                if (i < n) s.add(v);
                const bool keep = i < n && v != 1.0f;
                const uint32_t bk = __ballot_sync(0xFFFFFFFFu, keep);
                if (keep) {
                    vals[nv + __popc(bk & ((1u << lane) - 1u))] = v;
                    mn = fminf(mn, v);
                    mx = fmaxf(mx, v);
                }
                nv += __popc(bk);
                nb += __popc(__ballot_sync(0xFFFFFFFFu, i < n && v < 1.0f));
            }
            __syncwarp();
            o0 = warp_csum(s) / (float)n;
            const int n1 = n - nv;
            float os[4];
            int rv[4];
            bool one[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                one[q] = rk[q] >= nb && rk[q] < nb + n1;
                rv[q] = one[q] ? 0 : (rk[q] < nb ? rk[q] : rk[q] - n1);
            }
            if (nv > 0 && !(one[0] && one[1] && one[2] && one[3])) warp_order4(vals, nv, rv, hist, lane, mn, mx, os);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (one[q]) os[q] = 1.0f;
            o1 = fmaf(fr[0], os[1] - os[0], os[0]);
            o2 = fmaf(fr[1], os[3] - os[2], os[2]);
            __syncwarp();
        }
        if (lane == 0) {
            mean[j * Q.T + m] = o0;
            lo[j * Q.T + m] = o1;
            hi[j * Q.T + m] = o2;
        }
    }
}

int fill_segs(const int64_t* off, int M, Segs* s) {
    VPET_ARG(off, "model offsets: null pointer");
    VPET_ARG(M >= 1 && M <= MAXM, "model count must be in 1..%d", MAXM);
    s->M = M;
    for (int m = 0; m <= M; ++m) {
        s->off[m] = off[m];
        if (m > 0) VPET_ARG(off[m] >= off[m - 1], "model offsets must be non-decreasing");
    }
    return ABC_OK;
}

}  // namespace

extern "C" int abc_model_select(const int32_t* idx_dev, int64_t J, int32_t k, const int64_t* model_offsets_host,
                                int32_t M, float* prob_dev, int8_t* preferred_dev, void* stream) {
    vpet::clear_error();
    Segs S;
    int rc = fill_segs(model_offsets_host, M, &S);
    if (rc) return rc;
    VPET_ARG(J >= 0 && k >= 1, "abc_model_select: need J >= 0, k >= 1");
    if (J == 0) return ABC_OK;
    VPET_ARG(idx_dev && prob_dev && preferred_dev, "abc_model_select: null pointer");
    k_model_select<<<(unsigned)vpet_ceil_div(J, 8), 256, 0, (cudaStream_t)stream>>>(idx_dev, J, k, S, prob_dev,
                                                                                   preferred_dev);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

extern "C" int abc_summarize(const float* theta_dev, int32_t ldtheta, const int64_t* model_offsets_host, int32_t M,
                             const int32_t* nparams_host, const int32_t* has_ki_host, const int32_t* ki_cols_host,
                             const int32_t* idx_dev, int64_t J, int32_t k, const int8_t* preferred_dev, int32_t ncols,
                             float* mean_dev, float* sd_dev, float* lo_dev, float* hi_dev, void* stream) {
    vpet::clear_error();
    SumParams Q;
    memset(&Q, 0, sizeof Q);
    int rc = fill_segs(model_offsets_host, M, &Q.S);
    if (rc) return rc;
    VPET_ARG(nparams_host && has_ki_host && ki_cols_host, "abc_summarize: null host array");
    VPET_ARG(k >= 1 && k <= 2048, "abc_summarize: k must be in 1..2048");
    VPET_ARG(J >= 0, "abc_summarize: negative J");
    Q.Pmax = 0;
    for (int m = 0; m < M; ++m) {
        VPET_ARG(nparams_host[m] >= 1 && nparams_host[m] <= ldtheta, "abc_summarize: nparams out of range");
        Q.nparams[m] = nparams_host[m];
        Q.has_ki[m] = has_ki_host[m] != 0;
        if (nparams_host[m] > Q.Pmax) Q.Pmax = nparams_host[m];
        if (Q.has_ki[m])
            for (int c = 0; c < 3; ++c)
                VPET_ARG(ki_cols_host[c] >= 0 && ki_cols_host[c] < nparams_host[m], "abc_summarize: bad ki_cols");
    }
    for (int c = 0; c < 3; ++c) Q.ki[c] = ki_cols_host[c] < 0 ? 0 : ki_cols_host[c];
    VPET_ARG(ncols == Q.Pmax + 1, "abc_summarize: ncols must be max(nparams) + 1 = %d", Q.Pmax + 1);
    Q.ncols = ncols;
    Q.k = k;
    Q.ldt = ldtheta;
    int p2 = 32;
    while (p2 < k) p2 <<= 1;
    Q.p2 = p2;
    if (J == 0) return ABC_OK;
    VPET_ARG(theta_dev && idx_dev && mean_dev && sd_dev && lo_dev && hi_dev, "abc_summarize: null pointer");
    // row mode where a warp's table of accepted rows is small (at most 8 parameters, at most
    // 9 KB with the histogram: a block of up to 6 such warps stays within 48 KB, and an SM still
    // holds about 30 warps); otherwise the per-column gather
    const size_t row_bytes = (size_t)ncols * p2 * 4 + 1024;
    const bool rows = Q.Pmax <= 8 && row_bytes <= 9 * 1024;
    const bool vec4 = ((uintptr_t)theta_dev & 15u) == 0 && (ldtheta & 3) == 0;
    const size_t per_warp = rows ? row_bytes : (size_t)p2 * 8 + 1024;
    int warps = 8;
    while (warps > 1 && (size_t)warps * per_warp > 48 * 1024) warps = rows ? warps - 1 : warps >> 1;
    const size_t smem = (size_t)warps * per_warp;
    if (rows)
        k_summarize<true><<<(unsigned)vpet_ceil_div(J, warps), warps * 32, smem, (cudaStream_t)stream>>>(
            theta_dev, idx_dev, J, preferred_dev, Q, mean_dev, sd_dev, lo_dev, hi_dev, vec4);
    else
        k_summarize<false><<<(unsigned)vpet_ceil_div(J, warps), warps * 32, smem, (cudaStream_t)stream>>>(
            theta_dev, idx_dev, J, preferred_dev, Q, mean_dev, sd_dev, lo_dev, hi_dev, vec4);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

extern "C" int abc_response_cri(const float* theta_dev, int32_t ldtheta, const int32_t* idx_dev, int64_t J,
                                int32_t k, int64_t first, int64_t last, const float* t_host, int32_t T,
                                float* mean_dev, float* lo_dev, float* hi_dev, void* stream) {
    vpet::clear_error();
    VPET_ARG(ldtheta >= 7, "abc_response_cri: ldtheta must hold the 7 lp-ntPET parameters");
    VPET_ARG(k >= 1 && k <= 2048, "abc_response_cri: k must be in 1..2048");
    VPET_ARG(J >= 0, "abc_response_cri: negative J");
    VPET_ARG(first >= 0 && first <= last, "abc_response_cri: need 0 <= first <= last");
    VPET_ARG(T >= 1 && T <= RESP_MAXT, "abc_response_cri: T must be in 1..%d", RESP_MAXT);
    VPET_ARG(t_host, "abc_response_cri: null time grid");
    RespParams Q;
    memset(&Q, 0, sizeof Q);
    Q.first = first;
    Q.last = last;
    Q.ldt = ldtheta;
    Q.k = k;
    Q.T = T;
    for (int m = 0; m < T; ++m) {
        VPET_ARG(t_host[m] == t_host[m], "abc_response_cri: time %d is NaN", m);
        Q.t[m] = t_host[m];
    }
    int p2 = 32;
    while (p2 < k) p2 <<= 1;
    Q.p2 = p2;
    if (J == 0) return ABC_OK;
    VPET_ARG(theta_dev && idx_dev && mean_dev && lo_dev && hi_dev, "abc_response_cri: null pointer");
    const size_t per_warp = (size_t)p2 * 5 * 4 + 1024;
    int warps = 8;
    while (warps > 1 && (size_t)warps * per_warp > 96 * 1024) warps >>= 1;
    const size_t smem = (size_t)warps * per_warp;
    if (smem > 48 * 1024)
        VPET_CUDA(cudaFuncSetAttribute(k_response_cri, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_response_cri<<<(unsigned)vpet_ceil_div(J, warps), warps * 32, smem, (cudaStream_t)stream>>>(
        theta_dev, idx_dev, J, Q, mean_dev, lo_dev, hi_dev);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}
