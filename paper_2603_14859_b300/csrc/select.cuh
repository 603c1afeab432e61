// Warp-cooperative selection on per-voxel candidate lists (Algorithm 1, step 5:
// keep the smallest distances).  Candidates live in global memory as parallel
// arrays of fp32 keys and int32 draw indices; one warp works on one list.
#pragma once
#include <stdint.h>

namespace vpet {

// Order-preserving map of fp32 onto uint32 (negative values flipped).
__device__ __forceinline__ uint32_t f2key(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// Radix select over keys[0..cnt): returns a key value T with
//   #{i : key(keys[i]) <= T} >= rank + 1,
// resolved to the top `levels` x 8 bits (the returned T is the largest key of
// the bucket holding the element of that rank; levels = 4 gives the exact key).
// hist: 256 words of this warp's shared memory.  All lanes get the result.
__device__ __forceinline__ uint32_t warp_select(const float* keys, int cnt, int rank, int levels, uint32_t* hist,
                                                int lane) {
    uint32_t prefix = 0;
    int r = rank;
    for (int lv = 0; lv < levels; ++lv) {
        const int shift = 24 - 8 * lv;
        const uint32_t mask = lv == 0 ? 0u : (0xFFFFFFFFu << (shift + 8));
#pragma unroll
        for (int b = 0; b < 8; ++b) hist[lane * 8 + b] = 0;
        __syncwarp();
        // lanes holding the same bin are merged with match.any, so a bin that most
        // keys share costs one shared-memory atomic per 32 keys, not 32
        for (int base = 0; base < cnt; base += 128) {
            uint32_t kk[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = base + 32 * u + lane;
                kk[u] = i < cnt ? f2key(keys[i]) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool in = base + 32 * u + lane < cnt && (kk[u] & mask) == prefix;
                const uint32_t bin = (kk[u] >> shift) & 255u;
                const uint32_t peers = __match_any_sync(0xFFFFFFFFu, in ? bin : (0x100u | (uint32_t)lane));
                if (in && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
            }
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
        int found = -1, newr = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            if (found < 0 && c + loc[b] > (uint32_t)r) { found = lane * 8 + b; newr = r - (int)c; }
            c += loc[b];
        }
        const uint32_t who = __ballot_sync(0xFFFFFFFFu, found >= 0);
        const int src = who ? __ffs(who) - 1 : 31;
        const int bin = __shfl_sync(0xFFFFFFFFu, found, src);
        r = __shfl_sync(0xFFFFFFFFu, newr, src);
        prefix |= (uint32_t)(bin < 0 ? 255 : bin) << shift;
        __syncwarp();
    }
    const int low_bits = 32 - 8 * levels;
    return low_bits > 0 ? (prefix | ((1u << low_bits) - 1u)) : prefix;
}

// Cut for "at least the rank + 1 smallest" without an exact selection: 256
// equal-width bins over [min, max] of keys[0..cnt) (bin(v) = floor((v - min) *
// scale), monotone in v), and the bin b that holds the element of that rank.
// Keeping every key with bin(key) <= b keeps at least rank + 1 keys, and every
// dropped key exceeds every kept one.  Two passes (range, histogram) instead of
// one per radix digit.  hist: 256 words of this warp's shared memory.
struct LinearCut {
    float mn, scale;
    int bin;
    int below, inbin;   // keys in the bins below `bin`, and in `bin`
};

__device__ __forceinline__ int linear_bin(float v, const LinearCut& c) {
    const float t = (v - c.mn) * c.scale;
    return t < 255.0f ? (int)t : 255;
}

// Logical entry i of a list stored as two segments, [0, c0) and [off1, off1 + cnt - c0)
// (off1 >= c0; one segment when c0 >= cnt).
__device__ __forceinline__ int seg_pos(int i, int c0, int off1) { return i < c0 ? i : off1 + (i - c0); }

__device__ __forceinline__ LinearCut warp_cut_linear(const float* keys, int cnt, int rank, uint32_t* hist, int lane,
                                                     int c0 = 0x7FFFFFFF, int off1 = 0) {
    float mn = 3.0e38f, mx = -3.0e38f;
    for (int i = lane; i < cnt; i += 32) {
        const float v = keys[seg_pos(i, c0, off1)];
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    }
    LinearCut c;
    c.mn = mn;
    const float span = mx - mn;
    c.scale = span > 0.0f && span < 3.0e38f ? 256.0f / span : 0.0f;
    c.bin = 255;
    c.below = 0;
    c.inbin = cnt;
    if (c.scale == 0.0f) return c;          // one distinct value (or an unbounded range): keep all
#pragma unroll
    for (int b = 0; b < 8; ++b) hist[lane * 8 + b] = 0;
    __syncwarp();
    for (int base = 0; base < cnt; base += 128) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = base + 32 * u + lane;
            v[u] = i < cnt ? keys[seg_pos(i, c0, off1)] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (base + 32 * u + lane < cnt) atomicAdd(&hist[linear_bin(v[u], c)], 1u);
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
    uint32_t cum = incl - sum;
    int found = -1, below = 0, inbin = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if (found < 0 && cum + loc[b] > (uint32_t)rank) { found = lane * 8 + b; below = (int)cum; inbin = (int)loc[b]; }
        cum += loc[b];
    }
    const uint32_t who = __ballot_sync(0xFFFFFFFFu, found >= 0);
    const int src = who ? __ffs(who) - 1 : 0;
    c.bin = who ? __shfl_sync(0xFFFFFFFFu, found, src) : 255;
    c.below = who ? __shfl_sync(0xFFFFFFFFu, below, src) : 0;
    c.inbin = who ? __shfl_sync(0xFFFFFFFFu, inbin, src) : cnt;
    __syncwarp();
    return c;
}

// The k-th key with the number of keys strictly below it and equal to it.
struct KthKey {
    uint32_t K;
    int n_less, n_eq;
};

__device__ __forceinline__ KthKey warp_count_key(const float* keys, int cnt, uint32_t K, int lane) {
    int lt = 0, eq = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        const uint32_t k = i < cnt ? f2key(keys[i]) : 0xFFFFFFFFu;
        lt += __popc(__ballot_sync(0xFFFFFFFFu, i < cnt && k < K));
        eq += __popc(__ballot_sync(0xFFFFFFFFu, i < cnt && k == K));
    }
    return KthKey{K, lt, eq};
}

// Exact key of the given rank (0-based) among keys[0..cnt): the linear cut finds
// the bin holding it; that bin's keys (at most cap of them) are gathered into
// buf (this warp's shared memory) and the one of rank rank - below among them is
// found by counting, for each, the gathered keys below and equal to it.  A bin
// with more than cap keys falls back to the four-digit radix select.  Returns
// the order-preserving integer image of the key (as warp_select with 4 levels)
// and the counts of keys below and equal to it.
__device__ __forceinline__ KthKey warp_select_exact(const float* keys, int cnt, int rank, uint32_t* hist,
                                                    float* buf, int cap, int lane) {
    const LinearCut c = warp_cut_linear(keys, cnt, rank, hist, lane);
    if (c.scale == 0.0f) {
        // a single distinct value, or a range too wide for fp32 bins
        float mn = 3.0e38f, mx = -3.0e38f;
        for (int i = lane; i < cnt; i += 32) { mn = fminf(mn, keys[i]); mx = fmaxf(mx, keys[i]); }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
        }
        if (mn == mx) return KthKey{f2key(mn), 0, cnt};
        return warp_count_key(keys, cnt, warp_select(keys, cnt, rank, 4, hist, lane), lane);
    }
    if (c.inbin > cap) return warp_count_key(keys, cnt, warp_select(keys, cnt, rank, 4, hist, lane), lane);
    int m = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        const float v = i < cnt ? keys[i] : 0.0f;
        const bool in = i < cnt && linear_bin(v, c) == c.bin;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, in);
        if (in) buf[m + __popc(bal & ((1u << lane) - 1u))] = v;
        m += __popc(bal);
    }
    __syncwarp();
    const int r = rank - c.below;
    uint32_t K = 0u;
    int nlt = 0, neq = 0;
    bool got = false;
    for (int a = lane; a < m; a += 32) {
        const float v = buf[a];
        int lt = 0, eq = 0;
        for (int b = 0; b < m; ++b) {
            const float u = buf[b];
            lt += u < v;
            eq += u == v;
        }
        if (lt <= r && r < lt + eq) { K = f2key(v); nlt = lt; neq = eq; got = true; }
    }
    const uint32_t who = __ballot_sync(0xFFFFFFFFu, got);
    const int src = who ? __ffs(who) - 1 : 0;
    K = __shfl_sync(0xFFFFFFFFu, K, src);
    nlt = __shfl_sync(0xFFFFFFFFu, nlt, src);
    neq = __shfl_sync(0xFFFFFFFFu, neq, src);
    __syncwarp();
    return KthKey{K, c.below + nlt, neq};
}

// Radix select over the draw indices (non-negative int32) of the entries whose
// key equals K: the index of the given rank among them.  hist: 256 words.
__device__ __forceinline__ uint32_t warp_select_tie_index(const float* keys, const int32_t* idx, int cnt, uint32_t K,
                                                          int rank, uint32_t* hist, int lane) {
    uint32_t prefix = 0;
    int r = rank;
    for (int lv = 0; lv < 4; ++lv) {
        const int shift = 24 - 8 * lv;
        const uint32_t mask = lv == 0 ? 0u : (0xFFFFFFFFu << (shift + 8));
#pragma unroll
        for (int b = 0; b < 8; ++b) hist[lane * 8 + b] = 0;
        __syncwarp();
        for (int base = 0; base < cnt; base += 32) {
            const int i = base + lane;
            const uint32_t v = i < cnt ? (uint32_t)idx[i] : 0u;
            const bool in = i < cnt && f2key(keys[i]) == K && (v & mask) == prefix;
            const uint32_t bin = in ? (v >> shift) & 255u : (0x100u | (uint32_t)lane);
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, bin);
            if (in && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
        }
        __syncwarp();
        uint32_t loc[8], sum = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) { loc[b] = hist[lane * 8 + b]; sum += loc[b]; }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        uint32_t cum = incl - sum;
        int found = -1, newr = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            if (found < 0 && cum + loc[b] > (uint32_t)r) { found = lane * 8 + b; newr = r - (int)cum; }
            cum += loc[b];
        }
        const uint32_t who = __ballot_sync(0xFFFFFFFFu, found >= 0);
        const int src = who ? __ffs(who) - 1 : 31;
        const int bin = __shfl_sync(0xFFFFFFFFu, found, src);
        r = __shfl_sync(0xFFFFFFFFu, newr, src);
        prefix |= (uint32_t)(bin < 0 ? 255 : bin) << shift;
        __syncwarp();
    }
    return prefix;
}

// In-place stable compaction to the entries with key < K, or key == K and index <= Ti.
__device__ __forceinline__ int warp_compact_ties(float* keys, int32_t* idx, int cnt, uint32_t K, uint32_t Ti,
                                                 int lane) {
    int out = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        float k = 0.0f;
        int32_t id = 0;
        bool keep = false;
        if (i < cnt) {
            k = keys[i];
            id = idx[i];
            const uint32_t kk = f2key(k);
            keep = kk < K || (kk == K && (uint32_t)id <= Ti);
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
        const int pos = out + __popc(bal & ((1u << lane) - 1u));
        if (keep) {
            keys[pos] = k;
            idx[pos] = id;
        }
        out += __popc(bal);
    }
    __syncwarp();
    return out;
}

// In-place stable compaction of (keys, idx)[0..cnt) to the entries in bins <= c.bin;
// returns the number kept and (in kmax) the largest kept key.
__device__ __forceinline__ int warp_compact_cut(float* keys, int32_t* idx, int cnt, const LinearCut& c, int lane,
                                                float& kmax, int c0 = 0x7FFFFFFF, int off1 = 0) {
    int out = 0;
    float mx = -3.0e38f;
    // four rows of 32 read before any is written back: every write goes to a position
    // below the batch's first unread entry, so reading ahead is safe in place
    for (int base = 0; base < cnt; base += 128) {
        float k[4];
        int32_t id[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = base + 32 * u + lane;
            const int p = seg_pos(i, c0, off1);
            k[u] = i < cnt ? keys[p] : 0.0f;
            id[u] = i < cnt ? idx[p] : 0;
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = base + 32 * u + lane;
            const bool keep = i < cnt && linear_bin(k[u], c) <= c.bin;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
            const int pos = out + __popc(bal & ((1u << lane) - 1u));
            if (keep) {
                keys[pos] = k[u];
                idx[pos] = id[u];
                mx = fmaxf(mx, k[u]);
            }
            out += __popc(bal);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    kmax = mx;
    __syncwarp();
    return out;
}

// In-place stable compaction of (keys, idx)[0..cnt) to the entries with key <= T.
// At most `cap` entries are written; returns the number that qualified (which
// may exceed cap).
__device__ __forceinline__ int warp_compact(float* keys, int32_t* idx, int cnt, uint32_t T, int cap, int lane) {
    int out = 0;
    // four rows of 32 read ahead (safe in place: writes land below the batch)
    for (int base = 0; base < cnt; base += 128) {
        float k[4];
        int32_t id[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = base + 32 * u + lane;
            k[u] = i < cnt ? keys[i] : 0.0f;
            id[u] = i < cnt ? idx[i] : 0;
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = base + 32 * u + lane;
            const bool keep = i < cnt && f2key(k[u]) <= T;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
            const int pos = out + __popc(bal & ((1u << lane) - 1u));
            if (keep && pos < cap) {
                keys[pos] = k[u];
                idx[pos] = id[u];
            }
            out += __popc(bal);
        }
    }
    __syncwarp();
    return out;
}

// Ascending bitonic sort of n (a power of two) 64-bit keys in this warp's shared memory.
// Bitonic sort of 32 NE 64-bit keys held in registers, lane L holding elements
// L NE .. L NE + NE - 1 in v[0 .. NE - 1]: ascending over the element index.  Strides below
// NE compare within a lane (compile-time register indices), larger ones exchange with lane
// L ^ (stride / NE) through shuffles, each lane keeping the minimum or the maximum.
template <int S, int NE>
__device__ __forceinline__ void bitonic_in_lane(unsigned long long (&v)[NE], int size, int lane) {
#pragma unroll
    for (int i = 0; i < NE; ++i) {
        if (i & S) continue;
        const int e = lane * NE + i;
        const bool up = (e & size) == 0;
        const unsigned long long a = v[i], b = v[i + S];
        const bool sw = (a > b) == up;
        v[i] = sw ? b : a;
        v[i + S] = sw ? a : b;
    }
}

template <int NE>
__device__ __forceinline__ void warp_bitonic_sort_regs(unsigned long long (&v)[NE], int lane) {
    constexpr int N = 32 * NE;
    for (int size = 2; size <= N; size <<= 1) {
        for (int stride = size >> 1; stride >= NE; stride >>= 1) {
            const int lm = stride / NE;
            const bool lower = (lane & lm) == 0;
#pragma unroll
            for (int i = 0; i < NE; ++i) {
                const bool up = ((lane * NE + i) & size) == 0;
                const unsigned long long p = __shfl_xor_sync(0xFFFFFFFFu, v[i], lm);
                const bool take_min = lower == up;
                v[i] = take_min ? (p < v[i] ? p : v[i]) : (p > v[i] ? p : v[i]);
            }
        }
        const int s0 = (size >> 1) < NE ? (size >> 1) : NE / 2;   // the largest in-lane stride
        if (NE >= 16 && s0 >= 8) bitonic_in_lane<(NE >= 16 ? 8 : 1), NE>(v, size, lane);
        if (NE >= 8 && s0 >= 4) bitonic_in_lane<(NE >= 8 ? 4 : 1), NE>(v, size, lane);
        if (NE >= 4 && s0 >= 2) bitonic_in_lane<(NE >= 4 ? 2 : 1), NE>(v, size, lane);
        if (s0 >= 1) bitonic_in_lane<1, NE>(v, size, lane);
    }
}

__device__ __forceinline__ void warp_bitonic_sort(unsigned long long* s, int n, int lane) {
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncwarp();
            for (int t = lane; t < (n >> 1); t += 32) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const unsigned long long a = s[lo], b = s[hi];
                if ((a > b) == up) {
                    s[lo] = b;
                    s[hi] = a;
                }
            }
        }
    }
    __syncwarp();
}

}  // namespace vpet
