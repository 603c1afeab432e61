// Learned proposal for local ABC (a build extra; the paper has no counterpart):
// a small MLP maps a voxel TAC to a truncated-Gaussian proposal over the
// 2TCM-irr parameters, and importance-weighted local ABC then draws a few
// thousand proposals per voxel instead of scanning a million prior draws.
//
//  * Network: features (L + 1) -> H -> H -> 2P with GELU, fp32 master weights
//    used rounded to bf16, fp32 accumulation.  Outputs (mu_p, log sigma_p) in
//    unit-box coordinates u = (theta - lo) / (hi - lo).
//  * Loss: mean truncated-normal negative log likelihood of the true u
//    (mu clamped to [-3, 4], log sigma to [-7, 2]); analytic backward; Adam.
//  * Training pairs: prior draws -> simulated TACs -> the Gaussian
//    decay-weighted noise model of Sec. III-A (abc_add_noise), all on the GPU.
//  * Local ABC: per voxel M proposals u ~ TN(mu, sigma) on [0, 1] by inverse
//    CDF, their TACs, the k nearest kept, weights prior / proposal = 1 / q(u)
//    normalised over the accepted set, weighted summaries.  The irreversible
//    2TCM (Eq. 1-2 with k4 = 0) has
//      C_t = Vb C_p + (1 - Vb) K1 / a [k3 (1 (*) C_p) + k2 (e^{-a t} (*) C_p)],
//    a = k2 + k3, so every frame mean is a fixed combination of G(0), G(a) and
//    the frame mean of C_p, G(a) = frame mean of e^{-a t} (*) C_p.  G is
//    tabulated once per scan (with abc_simulate) on a_i = a_max (i / (T-1))^2
//    and read back by the cubic Lagrange interpolant through four nodes; the
//    distance is evaluated as y.y - 2 y.x + x.x from weighted dot products of
//    y, C_p, G(0) and G(a_i), tabulated and interpolated the same way.
#include <cuda_bf16.h>
#include <string.h>

#include "common.cuh"
#include "select.cuh"
#include "tc_ptx.cuh"

using namespace vpet;

namespace {

constexpr int MAXL = 64;
constexpr int GT = 64;          // unit of the split-K slab space
constexpr int LA_THREADS = 512;
constexpr int LA_P = 4;         // K1, k2, k3, Vb
constexpr int LA_C = LA_P + 1;  // ... and K_i
constexpr int LA_KMAX = 256;
constexpr int LA_CAP = 1024;    // bracketed candidates kept for exact selection
constexpr int LA_PILOT = 1024;  // pilot sample that brackets the k-th distance

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}
__device__ __forceinline__ float nphi(float z) { return 0.39894228040143268f * expf(-0.5f * z * z); }

// P(a < Z < b), a < b, without cancellation in either tail.
__device__ __forceinline__ float norm_mass(float a, float b) {
    constexpr float r2 = 0.70710678118654752f;
    if (a > 0.0f) return 0.5f * (erfcf(a * r2) - erfcf(b * r2));
    if (b < 0.0f) return 0.5f * (erfcf(-b * r2) - erfcf(-a * r2));
    return 1.0f - 0.5f * (erfcf(-a * r2) + erfcf(b * r2));
}

// ------------------------------------------------------------------ features
struct FrameW {
    float w[MAXL];
};

// f_l = y_l / s (l < L), f_L = log(s) / 10, s = sqrt(sum_l w_l y_l^2) + 1e-30; one warp per voxel
__global__ void k_features(const float* __restrict__ y, int64_t J, int ldy, int L, FrameW W, float* __restrict__ f) {
    // the weights in shared memory: a lane-indexed read of the parameter space is serialised
    __shared__ float sw[MAXL];
    for (int l = threadIdx.x; l < L; l += blockDim.x) sw[l] = W.w[l];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= J) return;
    const float* yr = y + j * ldy;
    float ss = 0.0f;
    for (int l = lane; l < L; l += 32) ss = fmaf(sw[l] * yr[l], yr[l], ss);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
    const float s = sqrtf(ss) + 1e-30f;
    float* fr = f + j * (L + 1);
    for (int l = lane; l < L; l += 32) fr[l] = yr[l] / s;
    if (lane == 0) fr[L] = logf(s) * 0.1f;
}

// ------------------------------------------------------------------ GEMM
// C[m, n] = sum_k A(m, k) B(k, n) (+ bias[n]), A(m, k) = gelu?(A[m sam + k sak]),
// B(k, n) = gelu?/bf16?(B[k sbk + n sbn]), on the tensor cores (tcgen05, fp32 accumulators
// in TMEM).  The fp32 operands are split into bf16 parts: an activation (or gradient) into
// three, hi + mid + lo, which hold its 24 bits; a weight, rounded to bf16 at every use, is
// one part.  Products of parts are exact in fp32, so C equals the fp32 sum up to the
// accumulation's rounding: with a one-part B the three products hi.B, mid.B, lo.B; with
// two three-part operands the six whose weight is at least 2^-16 (hi.hi, hi.mid, mid.hi,
// hi.lo, mid.mid, lo.hi), leaving terms of order 2^-24 relative.  One CTA computes a
// 128 x BN tile: its 256 threads load a 64-wide K block of A and B, apply GELU / the
// rounding, split and store the parts in the 128-byte-swizzled K-major layout of the
// MMA's shared-memory descriptors (two stages, so loading one block overlaps the MMAs of
// the previous), and one thread issues the MMAs.  With split-K (gridDim.z > 1) each
// z-slice stores its partial sums in its own M x N slab and k_splitk_sum adds the slabs in
// z order, so the result does not depend on the order the blocks finish in.
struct GemmArgs {
    const float* A;
    int64_t sam, sak;
    const float* B;
    int64_t sbk, sbn;
    float* C;
    int64_t ldc;
    const float* bias;
    int M, N, K;
    int actA;    // 1 = GELU of the loaded A value
    int actB;    // 1 = GELU of the loaded B value
    int roundB;  // 1 = B rounded to bf16 (weights: one part)
    float* part = nullptr;     // split-K slabs (null: no split)
    int64_t part_cap = 0;      // floats available there
};

// floats of split-K slab space in the training workspace: enough for about
// three waves of 64 x 64 tiles on up to 192 SMs
constexpr int64_t GEMM_PART_FLOATS = 3LL * 192 * GT * GT;

constexpr int TC_M = 128;                       // tile rows (TMEM lanes)
constexpr int TC_KB = 64;                       // K per block: one 128-byte row of bf16
constexpr int TC_THREADS = 256;                 // 8 warps: two per TMEM lane quarter
constexpr int TC_APARTS = 3;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;  // bound on every barrier wait

struct TcGemm {
    GemmArgs g;
    int bn;                      // tile width in N (multiple of 16, <= 256)
    int pb;                      // parts of B: 1 (weights) or 3
    int kchunk;                  // K per z-slice (a multiple of TC_KB)
    int tmem_cols;
    int* err;                    // set when a bounded wait ran out
};

__device__ int g_mlp_timeout = 0;

// byte offset of element (r, k), k < 64, in a 128-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
    return (uint32_t)r * 128u + ((((uint32_t)k >> 3) ^ ((uint32_t)r & 7u)) << 4) + ((uint32_t)k & 7u) * 2u;
}

__device__ __forceinline__ void split3(float v, __nv_bfloat16 (&p)[3]) {
    p[0] = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(p[0]);
    p[1] = __float2bfloat16_rn(r1);
    p[2] = __float2bfloat16_rn(r1 - __bfloat162float(p[1]));
}

__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(const __grid_constant__ TcGemm T) {
    extern __shared__ __align__(1024) uint8_t tc_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    const GemmArgs& g = T.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bn = T.bn, pb = T.pb;
    const uint32_t a_bytes = TC_M * 128, b_bytes = (uint32_t)bn * 128;
    const uint32_t stage_bytes = TC_APARTS * a_bytes + (uint32_t)pb * b_bytes;
    const int64_t m0 = (int64_t)blockIdx.y * TC_M, n0 = (int64_t)blockIdx.x * bn;
    const int kbeg = blockIdx.z * T.kchunk, kend = min(g.K, kbeg + T.kchunk);
    const int nkb = (kend - kbeg + TC_KB - 1) / TC_KB;
    if (tid == 0) {
        ptx::mbar_init(ptx::smem_u32(&bar[0]), 1);
        ptx::mbar_init(ptx::smem_u32(&bar[1]), 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        ptx::tmem_alloc(ptx::smem_u32(&tmem_base), (uint32_t)T.tmem_cols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = ptx::idesc_bf16_f32(TC_M, bn);
    bool failed = false;
    int issued = -1;                             // last K block whose MMAs were issued
    for (int kb = 0; kb < nkb; ++kb) {
        const int st = kb & 1;
        uint8_t* sa = sm + st * stage_bytes;
        uint8_t* sb = sa + TC_APARTS * a_bytes;
        // the MMAs two blocks back read this stage
        bool ok = true;
        if (kb >= 2) ok = ptx::mbar_wait(ptx::smem_u32(&bar[st]), ((kb - 2) >> 1) & 1, TC_WAIT_NS);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const int k0 = kbeg + kb * TC_KB;
        // eight independent loads in flight per thread, then their GELU, split and stores
        constexpr int CH = 8;
        for (int e0 = tid; e0 < TC_M * TC_KB; e0 += TC_THREADS * CH) {
            float v[CH];
            uint32_t off[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int e = e0 + u * TC_THREADS;
                int r, kk;
                if (g.sak == 1) { r = e >> 6; kk = e & 63; } else { r = e & 127; kk = e >> 7; }
                const int64_t m = m0 + r;
                const int k = k0 + kk;
                off[u] = sw128_off(r, kk);
                v[u] = (m < g.M && k < kend) ? g.A[m * g.sam + (int64_t)k * g.sak] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                __nv_bfloat16 p[3];
                split3(g.actA ? gelu(v[u]) : v[u], p);
#pragma unroll
                for (int q = 0; q < 3; ++q) *(__nv_bfloat16*)(sa + q * a_bytes + off[u]) = p[q];
            }
        }
        for (int e0 = tid; e0 < bn * TC_KB; e0 += TC_THREADS * CH) {
            float v[CH];
            uint32_t off[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int e = e0 + u * TC_THREADS;
                int r, kk;
                if (g.sbk == 1) { r = e >> 6; kk = e & 63; } else { r = e % bn; kk = e / bn; }
                const int64_t n = n0 + r;
                const int k = k0 + kk;
                off[u] = e < bn * TC_KB ? sw128_off(r, kk) : 0xFFFFFFFFu;
                v[u] = (e < bn * TC_KB && n < g.N && k < kend) ? g.B[(int64_t)k * g.sbk + n * g.sbn] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if (off[u] == 0xFFFFFFFFu) continue;
                const float b = g.actB ? gelu(v[u]) : v[u];
                if (pb == 1) {
                    *(__nv_bfloat16*)(sb + off[u]) = __float2bfloat16_rn(b);
                } else {
                    __nv_bfloat16 p[3];
                    split3(b, p);
#pragma unroll
                    for (int q = 0; q < 3; ++q) *(__nv_bfloat16*)(sb + q * b_bytes + off[u]) = p[q];
                }
            }
        }
        // the generic-proxy stores must be visible to the tensor cores' async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            ptx::tc_fence_after();
            // (A part, B part) products: three with a one-part B, six with three parts
            const int np = pb == 1 ? 3 : 6;
            const int pa_of[6] = {0, 1, 2, 0, 1, 0}, pb_of[6] = {0, 0, 0, 1, 1, 2};
            for (int q = 0; q < np; ++q) {
                const uint32_t abase = ptx::smem_u32(sa + pa_of[q] * a_bytes);
                const uint32_t bbase = ptx::smem_u32(sb + (pb == 1 ? 0 : pb_of[q]) * b_bytes);
#pragma unroll
                for (int ks = 0; ks < TC_KB / 16; ++ks)
                    ptx::mma_bf16(tmem, ptx::desc_sw128(abase + ks * 32), ptx::desc_sw128(bbase + ks * 32), idesc,
                                  (kb > 0 || q > 0 || ks > 0) ? 1u : 0u);
            }
            ptx::mma_commit(ptx::smem_u32(&bar[st]));
        }
        issued = kb;
    }
    // the last commit covers every MMA this CTA issued
    if (issued >= 0) {
        const bool ok = ptx::mbar_wait(ptx::smem_u32(&bar[issued & 1]), (issued >> 1) & 1, TC_WAIT_NS);
        if (__syncthreads_or(!ok)) failed = true;
    }
    ptx::tc_fence_after();
    if (!failed && issued >= 0) {
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows), every other 32-column chunk
        const int quarter = warp & 3;
        const int64_t m = m0 + quarter * 32 + lane;
        for (int c0 = (warp >> 2) * 32; c0 < bn; c0 += 64) {
            uint32_t r[32];
            ptx::tmem_ld32_async(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, r);
            ptx::tmem_wait_ld();
            ptx::tmem_fence_regs(r);
            if (m < g.M) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int64_t n = n0 + c0 + i;
                    if (n >= g.N) break;
                    float v = __uint_as_float(r[i]);
                    if (gridDim.z > 1) {
                        g.part[((int64_t)blockIdx.z * g.M + m) * g.N + n] = v;
                    } else {
                        if (g.bias) v += g.bias[n];
                        g.C[m * g.ldc + n] = v;
                    }
                }
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, (uint32_t)T.tmem_cols);
    }
    if (failed && tid == 0) atomicExch(T.err, 1);
}

// C[m, n] = sum_z part[z, m, n] (+ bias[n]), z ascending
__global__ void k_splitk_sum(const float* __restrict__ part, int split, int M, int N, const float* __restrict__ bias,
                             float* __restrict__ C, int64_t ldc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t MN = (int64_t)M * N;
    if (e >= MN) return;
    const int m = (int)(e / N), n = (int)(e - (int64_t)m * N);
    float v = 0.0f;
    for (int z = 0; z < split; ++z) v += part[z * MN + e];
    if (bias) v += bias[n];
    C[(int64_t)m * ldc + n] = v;
}

int g_sms = 0;
size_t g_tc_smem_set = 0;
int* g_timeout_flag = nullptr;   // device address of g_mlp_timeout

int gemm(const GemmArgs& a, cudaStream_t s) {
    if (g_sms == 0) {
        int dev = 0;
        VPET_CUDA(cudaGetDevice(&dev));
        VPET_CUDA(cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    TcGemm T;
    T.g = a;
    T.pb = a.roundB ? 1 : 3;
    // a tile of 128 x bn; three-part B tiles are narrower so that two stages fit in shared memory
    int bn_max = T.pb == 1 ? 256 : 128;
    // narrower tiles when the wide ones would leave most SMs idle (the training batch)
    if (vpet_ceil_div(a.M, TC_M) * vpet_ceil_div(a.N, bn_max) < 2 * g_sms) bn_max = 64;
    const int64_t nr = vpet_round_up(a.N, 16);
    T.bn = (int)(nr < bn_max ? nr : bn_max);
    int cols = 32;
    while (cols < T.bn) cols <<= 1;
    T.tmem_cols = cols;
    if (!g_timeout_flag) VPET_CUDA(cudaGetSymbolAddress((void**)&g_timeout_flag, g_mlp_timeout));
    T.err = g_timeout_flag;
    const int64_t ntn = vpet_ceil_div(a.N, T.bn), ntm = vpet_ceil_div(a.M, TC_M);
    VPET_ARG(ntm <= 65535 && ntn <= 65535, "mlp: %d rows exceed one launch's grid (at most %d)", a.M, 65535 * TC_M);
    const int64_t tiles = ntn * ntm;
    // split K when the output has too few tiles to fill the GPU (weight gradients)
    int64_t split = 1;
    if (a.part && tiles < g_sms && a.K >= 8 * TC_KB) {
        split = vpet_ceil_div(2 * g_sms, tiles);
        const int64_t maxsplit = a.K / (4 * TC_KB);
        const int64_t capsplit = a.part_cap / ((int64_t)a.M * a.N);
        if (split > maxsplit) split = maxsplit;
        if (split > capsplit) split = capsplit;
        if (split < 1) split = 1;
    }
    T.kchunk = (int)vpet_round_up(vpet_ceil_div(a.K, split), TC_KB);
    split = vpet_ceil_div(a.K, T.kchunk);
    const size_t smem = 1024 + 2 * ((size_t)TC_APARTS * TC_M * 128 + (size_t)T.pb * T.bn * 128);
    if (smem > g_tc_smem_set) {
        VPET_CUDA(cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        g_tc_smem_set = smem;
    }
    const dim3 grid((unsigned)ntn, (unsigned)ntm, (unsigned)split);
    k_gemm_tc<<<grid, TC_THREADS, smem, s>>>(T);
    VPET_LAUNCH_CHECK();
    if (split > 1) {
        const int64_t MN = (int64_t)a.M * a.N;
        k_splitk_sum<<<(unsigned)vpet_ceil_div(MN, 256), 256, 0, s>>>(a.part, (int)split, a.M, a.N, a.bias, a.C,
                                                                      a.ldc);
        VPET_LAUNCH_CHECK();
    }
    return ABC_OK;
}

// dZ = dH * gelu'(Z)
__global__ void k_gelu_back(const float* __restrict__ dh, const float* __restrict__ z, float* __restrict__ dz,
                            int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dz[i] = dh[i] * gelu_d(z[i]);
}

// out[n] = sum_b X[b, n]: a block per 32 columns, rows split over its 8 warps
__global__ void k_colsum(const float* __restrict__ x, int B, int N, float* __restrict__ out) {
    __shared__ float part[8][33];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + lane;
    float s = 0.0f;
    if (n < N)
        for (int b = wp; b < B; b += 8) s += x[(int64_t)b * N + n];
    part[wp][lane] = s;
    __syncthreads();
    if (wp == 0 && n < N) {
        float t = 0.0f;
        for (int q = 0; q < 8; ++q) t += part[q][lane];
        out[n] = t;
    }
}

// truncated-normal NLL of targets T (B x P) under out (B x 2P); dout = d(mean NLL) / d(out)
__global__ void k_trunc_nll(const float* __restrict__ out, const float* __restrict__ T, int B, int P,
                            float* __restrict__ dout, float* __restrict__ loss) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (e < (int64_t)B * P) {
        const int64_t n = e / P;
        const int p = (int)(e - n * P);
        float mu = out[n * 2 * P + 2 * p], s = out[n * 2 * P + 2 * p + 1];
        const bool mu_in = mu >= -3.0f && mu <= 4.0f, s_in = s >= -7.0f && s <= 2.0f;
        mu = fminf(fmaxf(mu, -3.0f), 4.0f);
        s = fminf(fmaxf(s, -7.0f), 2.0f);
        const float sg = expf(s), t = T[e];
        const float z = (t - mu) / sg, a = -mu / sg, b = (1.0f - mu) / sg;
        const float Z = fmaxf(norm_mass(a, b), 1e-30f);
        l = s + 0.5f * z * z + logf(Z) + 0.91893853320467274f;
        const float dmu = -z / sg + (nphi(a) - nphi(b)) / (sg * Z);
        const float ds = 1.0f - z * z + (a * nphi(a) - b * nphi(b)) / Z;
        dout[n * 2 * P + 2 * p] = mu_in ? dmu / B : 0.0f;
        dout[n * 2 * P + 2 * p + 1] = s_in ? ds / B : 0.0f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / B);
}

// t[n, p] = (theta[n, p] - lo_p) / (hi_p - lo_p), clamped to [0, 1]
struct Box {
    float lo[8], inv[8];
};
__global__ void k_unit_box(const float* __restrict__ th, int64_t N, int ldt, int P, Box b, float* __restrict__ t) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * P) return;
    const int64_t n = e / P;
    const int p = (int)(e - n * P);
    t[e] = fminf(fmaxf((th[n * ldt + p] - b.lo[p]) * b.inv[p], 0.0f), 1.0f);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------------ Philox4x32-10 (Salmon et al., SC'11)
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}
// uniform in (0, 1) from the top 23 bits: ((r >> 9) + 1/2) 2^-23, exact in fp32
__device__ __forceinline__ float u01(uint32_t r) { return ((float)(r >> 9) + 0.5f) * 1.1920928955078125e-7f; }

// weights W ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)), zero biases
__global__ void k_mlp_init(float* p, int D, int H, int O, uint64_t seed) {
    const int64_t n1 = (int64_t)H * D, n2 = n1 + H, n3 = n2 + (int64_t)H * H, n4 = n3 + H, n5 = n4 + (int64_t)O * H,
                  n6 = n5 + O;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n6) return;
    float fan = 0.0f;
    if (i < n1) fan = (float)D;
    else if (i >= n2 && i < n3) fan = (float)H;
    else if (i >= n4 && i < n5) fan = (float)H;
    if (fan == 0.0f) { p[i] = 0.0f; return; }
    const uint4 r = philox(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0x6D6C70u, 0u), (uint32_t)seed,
                           (uint32_t)(seed >> 32));
    p[i] = (2.0f * u01(r.x) - 1.0f) * rsqrtf(fan);
}

// Gaussian decay-weighted noise (Sec. III-A): y = x + l_n sigma z with
// sigma_l = sqrt(max(x_l, 0) exp(lambda t_mid,l) / dt_l), l_n = q ||x|| / ||sigma||,
// q ~ U(q_lo, q_hi), z ~ N(0, 1) by Box-Muller on Philox uniforms; one warp per row.
struct NoiseFrames {
    int L;
    float tmid[MAXL];
    float dt[MAXL];
};

__global__ void k_add_noise(const float* __restrict__ x, int64_t N, int ldx, NoiseFrames F, float lambda, float q_lo,
                            float q_hi, uint64_t seed, int64_t first, float* __restrict__ y, int ldy) {
    __shared__ float s_tmid[MAXL], s_dt[MAXL];
    for (int l = threadIdx.x; l < F.L; l += blockDim.x) {
        s_tmid[l] = F.tmid[l];
        s_dt[l] = F.dt[l];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t n = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (n >= N) return;
    const uint64_t g = (uint64_t)(first + n);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const float* xr = x + n * ldx;
    float sx = 0.0f, ss = 0.0f, sig[2] = {0.0f, 0.0f}, z[2] = {0.0f, 0.0f}, xv[2] = {0.0f, 0.0f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int l = lane + 32 * h;
        if (l >= F.L) continue;
        xv[h] = xr[l];
        const float s = sqrtf(fmaxf(xv[h], 0.0f) * expf(lambda * s_tmid[l]) / s_dt[l]);
        sig[h] = s;
        sx = fmaf(xv[h], xv[h], sx);
        ss = fmaf(s, s, ss);
        const uint4 r = philox(make_uint4((uint32_t)g, (uint32_t)(g >> 32), 0x4E4F49u, (uint32_t)l), k0, k1);
        z[h] = sqrtf(-2.0f * logf(u01(r.x))) * cospif(2.0f * u01(r.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xFFFFFFFFu, sx, o);
        ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
    }
    const uint4 rq = philox(make_uint4((uint32_t)g, (uint32_t)(g >> 32), 0x515556u, 0u), k0, k1);
    const float q = q_lo + (q_hi - q_lo) * u01(rq.x);
    const float ln = ss > 0.0f ? q * sqrtf(sx) / sqrtf(ss) : 0.0f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int l = lane + 32 * h;
        if (l < F.L) y[n * ldy + l] = xv[h] + ln * sig[h] * z[h];
    }
}

// ------------------------------------------------------------------ local importance-weighted ABC
struct LocalArgs {
    const float* y;
    int64_t J;
    int ldy, L;
    float w[MAXL];
    const float* prop;     // J x 2P network outputs (mu, log sigma) per parameter
    const float* table;    // L x T, frame-major: column i = G(a_i); column 0 = G(0) = frame means of 1 (*) C_p
    const float* cpf;      // L frame means of C_p
    int T;
    int n_pilot, r_lo, r_hi;  // pilot sample size (0: no bracketing) and the ranks of its two pivots
    float a_max;
    float lo[LA_P], hi[LA_P];
    int M, k;
    float sigma_scale;     // proposal widening: sigma = sigma_scale exp(clamped log sigma)
    uint64_t seed;
    float* mean;           // J x 5: K1, k2, k3, Vb, K_i
    float* sd;
    float* qlo;
    float* qhi;
    float* ess;            // J
    float* dmed;           // J: median accepted distance
    float* ynorm;          // J: sum_l w_l y_l^2
    float* u_dump;         // optional J x M x P proposals (tests)
    float* d_dump;         // optional J x M distances (tests)
};

struct TnParams {         // truncated normal on [0, 1], per voxel and parameter
    float mu, sg, lnorm;  // lnorm = log sigma + log Z + log sqrt(2 pi)
    float pa, pb;         // CDF at the bounds, taken in the tail where it is accurate
    float sgs;            // sg, negated when pa, pb are upper-tail probabilities
};

__device__ __forceinline__ TnParams tn_params(float mu_raw, float s_raw, float sigma_scale) {
    TnParams t;
    t.mu = fminf(fmaxf(mu_raw, -3.0f), 4.0f);
    const float s = fminf(fmaxf(s_raw, -7.0f), 2.0f) + logf(sigma_scale);
    t.sg = expf(s);
    const float a = -t.mu / t.sg, b = (1.0f - t.mu) / t.sg;
    t.lnorm = s + logf(fmaxf(norm_mass(a, b), 1e-30f)) + 0.91893853320467274f;
    const bool upper = a + b > 0.0f;
    if (upper) { t.pa = normcdff(-a); t.pb = normcdff(-b); }
    else { t.pa = normcdff(a); t.pb = normcdff(b); }
    t.sgs = upper ? -t.sg : t.sg;
    return t;
}

// inverse-CDF draw: u uniform in (0, 1) -> t in [0, 1]
__device__ __forceinline__ float tn_draw(const TnParams& t, float u) {
    // pa (1 - u) + pb u: two non-negative terms (1 - u is exact for these uniforms), no cancellation
    const float p = fminf(fmaxf(fmaf(t.pa, 1.0f - u, u * t.pb), 1e-30f), 1.0f - 6e-8f);
    const float zq = normcdfinvf(p);
    const float v = fmaf(t.sgs, zq, t.mu);
    return fminf(fmaxf(v, 0.0f), 1.0f);
}

__device__ __forceinline__ float tn_logpdf(const TnParams& t, float v) {
    const float z = (v - t.mu) / t.sg;
    return -0.5f * z * z - t.lnorm;
}

// the P proposal coordinates of proposal i of voxel j
__device__ __forceinline__ void draw_u(const LocalArgs& A, const TnParams* tp, int64_t j, int i, float* u) {
    const uint4 r = philox(make_uint4((uint32_t)i, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), 0x4C4F43u),
                           (uint32_t)A.seed, (uint32_t)(A.seed >> 32));
    u[0] = tn_draw(tp[0], u01(r.x));
    u[1] = tn_draw(tp[1], u01(r.y));
    u[2] = tn_draw(tp[2], u01(r.z));
    u[3] = tn_draw(tp[3], u01(r.w));
}

// One warp: the bin of hist[256] that holds the key of rank r (0-based) and that
// key's rank within the bin.
__device__ __forceinline__ void warp_find_bin(const uint32_t* hist, int r, int lane, int* bin_out, int* r_out) {
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
    const int nr = __shfl_sync(0xFFFFFFFFu, newr, src);
    if (lane == 0) { *bin_out = bin < 0 ? 255 : bin; *r_out = nr; }
}

// Block-wide radix select (8-bit digits, most significant first) of two ranks at
// once over n fp32 keys in shared memory: out[q] = the exact key of rank rank[q]
// (0-based), ties[q] = its rank among the keys equal to it (rank minus the
// number of keys strictly below).  Lanes with the same digit add their count
// once (the keys of one voxel share few leading digits, so per-key atomics
// would queue on a handful of bins).  h holds 2 x 256 counters.
__device__ void block_select2(const float* keys, int n, int rank0, int rank1, uint32_t* h, int* sh, uint32_t* out,
                              int* ties) {
    uint32_t p0 = 0, p1 = 0;
    int r0 = rank0, r1 = rank1;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int lv = 0; lv < 4; ++lv) {
        const int shift = 24 - 8 * lv;
        const uint32_t mask = lv == 0 ? 0u : (0xFFFFFFFFu << (shift + 8));
        for (int b = threadIdx.x; b < 512; b += blockDim.x) h[b] = 0;
        __syncthreads();
        for (int i0 = 0; i0 < n; i0 += blockDim.x) {
            const int i = i0 + threadIdx.x;
            const uint32_t k = i < n ? f2key(keys[i]) : 0u;
            const uint32_t d = (k >> shift) & 255u;
            const uint32_t b0 = (i < n && (k & mask) == p0) ? d : 256u;
            const uint32_t b1 = (i < n && (k & mask) == p1) ? d : 256u;
            const uint32_t s0 = __match_any_sync(0xFFFFFFFFu, b0);
            if (b0 < 256u && lane == __ffs(s0) - 1) atomicAdd(&h[b0], (uint32_t)__popc(s0));
            const uint32_t s1 = __match_any_sync(0xFFFFFFFFu, b1);
            if (b1 < 256u && lane == __ffs(s1) - 1) atomicAdd(&h[256 + b1], (uint32_t)__popc(s1));
        }
        __syncthreads();
        if (wp < 2) warp_find_bin(h + 256 * wp, wp ? r1 : r0, lane, &sh[2 * wp], &sh[2 * wp + 1]);
        __syncthreads();
        p0 |= (uint32_t)sh[0] << shift;
        r0 = sh[1];
        p1 |= (uint32_t)sh[2] << shift;
        r1 = sh[3];
        __syncthreads();
    }
    out[0] = p0;
    out[1] = p1;
    if (ties) { ties[0] = r0; ties[1] = r1; }
}

__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.0f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    return t;
}

__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = -3.0e38f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = fmaxf(t, red[q]);
    return t;
}

// Persistent blocks over voxels.  Per voxel: M proposals and their distances (a
// quadratic form in three TAC coefficients over tabulated dot products), the
// exact k-th distance (a pilot sample brackets it; exact selection runs over
// the bracketed candidates, or over all keys when the bracket misses), ordered
// compaction of the accepted set (ties at the k-th distance to the lower
// proposal index), importance weights, weighted moments and weighted
// quantiles (bisection on the value order, one warp per column).
__global__ void __launch_bounds__(LA_THREADS, 2) k_local_abc(LocalArgs A) {
    extern __shared__ __align__(16) uint8_t sm[];
    float4* qt = (float4*)sm;                             // T: (y . G(a_i) per voxel, cp . G(a_i), G(0) . G(a_i),
                                                          //     G(a_i) . G(a_i)), all frame-weighted
    float* cps = (float*)(qt + A.T);                      // MAXL
    float* ys = cps + MAXL;                               // MAXL
    float* keys = ys + MAXL;                              // max(M, LA_C LA_KMAX): distances, then the
    float* sv = keys;                                     //   LA_C x LA_KMAX accepted values
    const int kreg = A.M > LA_C * LA_KMAX ? A.M : LA_C * LA_KMAX;
    int32_t* acc = (int32_t*)(keys + kreg);               // LA_KMAX accepted proposal indices
    float* wacc = (float*)(acc + LA_KMAX);                // LA_KMAX normalised weights
    float* red = wacc + LA_KMAX;                          // 64
    uint32_t* hist = (uint32_t*)(red + 64);               // 2 x 256
    int* sh = (int*)(hist + 512);                         // 8
    int* wcnt = sh + 8;                                   // 2 x 16 warp counts
    float* scal = (float*)(wcnt + 32);                    // 8: cp . cp, y . y, y . cp
    float* ckey = scal + 8;                               // LA_CAP candidate keys
    int32_t* cidx = (int32_t*)(ckey + LA_CAP);            // LA_CAP candidate proposal indices
    __shared__ TnParams tp[LA_P];
    const float* G = A.table;                             // L x T, frame-major

    for (int l = threadIdx.x; l < A.L; l += blockDim.x) cps[l] = A.cpf[l];
    __syncthreads();
    // With x = alpha cp + beta G(0) + gamma G(a) (alpha = Vb, beta = (1 - Vb) K1 k3 / a,
    // gamma = (1 - Vb) K1 k2 / a), d = sum_l w_l (y_l - x_l)^2 is a quadratic form in
    // (alpha, beta, gamma) whose coefficients are weighted dot products of y, cp, G(0) and
    // G(a).  The ones involving G(a) are tabulated on the a_i grid (per block, and y . G(a_i)
    // per voxel) and interpolated like G itself (the products are linear in G, or smooth).
    for (int i = threadIdx.x; i < A.T; i += blockDim.x) {
        float a = 0.0f, b = 0.0f, c = 0.0f;
        for (int l = 0; l < A.L; ++l) {
            const float g = G[(size_t)l * A.T + i];
            const float wr = A.w[l] * g;
            a = fmaf(wr, cps[l], a);
            b = fmaf(wr, G[(size_t)l * A.T], b);
            c = fmaf(wr, g, c);
        }
        qt[i] = make_float4(0.0f, a, b, c);
    }
    if (threadIdx.x == 0) {
        float cc = 0.0f;
        for (int l = 0; l < A.L; ++l) cc = fmaf(A.w[l] * cps[l], cps[l], cc);
        scal[0] = cc;
    }
    const float scale = (float)(A.T - 1) * rsqrtf(A.a_max);
    const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const uint32_t below = (1u << lane) - 1u;
    const int seg = (A.M + nw - 1) / nw;                  // warp wp owns proposals [s0, s1)
    const int s0 = min(A.M, wp * seg), s1 = min(A.M, s0 + seg);

    for (int64_t j = blockIdx.x; j < A.J; j += gridDim.x) {
        __syncthreads();
        for (int l = threadIdx.x; l < A.L; l += blockDim.x) ys[l] = A.y[j * A.ldy + l];
        if (threadIdx.x < LA_P)
            tp[threadIdx.x] = tn_params(A.prop[j * 2 * LA_P + 2 * threadIdx.x],
                                        A.prop[j * 2 * LA_P + 2 * threadIdx.x + 1], A.sigma_scale);
        if (threadIdx.x == 0) sh[4] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < A.T; i += blockDim.x) {
            float a = 0.0f;
            for (int l = 0; l < A.L; ++l) a = fmaf(A.w[l] * ys[l], G[(size_t)l * A.T + i], a);
            qt[i].x = a;
        }
        if (threadIdx.x == 0) {
            float yy = 0.0f, yc = 0.0f;
            for (int l = 0; l < A.L; ++l) {
                yy = fmaf(A.w[l] * ys[l], ys[l], yy);
                yc = fmaf(A.w[l] * ys[l], cps[l], yc);
            }
            scal[1] = yy;
            scal[2] = yc;
        }
        __syncthreads();
        const float4 q00 = qt[0];
        const float cc = scal[0], yy = scal[1], yc = scal[2], yg0 = q00.x, cg0 = q00.y, g00 = q00.w;

        // proposals, their TACs and distances
        for (int i = threadIdx.x; i < A.M; i += blockDim.x) {
            float u[LA_P];
            draw_u(A, tp, j, i, u);
            const float K1 = A.lo[0] + (A.hi[0] - A.lo[0]) * u[0];
            const float k2 = A.lo[1] + (A.hi[1] - A.lo[1]) * u[1];
            const float k3 = A.lo[2] + (A.hi[2] - A.lo[2]) * u[2];
            const float Vb = A.lo[3] + (A.hi[3] - A.lo[3]) * u[3];
            const float a = k2 + k3;
            const float pos = scale * sqrtf(fminf(fmaxf(a, 0.0f), A.a_max));
            const int i0 = max(1, min((int)pos, A.T - 3));
            const float t = pos - (float)i0;
            // Lagrange basis on the nodes i0-1, i0, i0+1, i0+2
            const float tm = t - 1.0f, tp1 = t + 1.0f, t2 = t - 2.0f;
            const float c0 = -t * tm * t2 * (1.0f / 6.0f), c1 = 0.5f * tp1 * tm * t2, c2 = -0.5f * tp1 * t * t2,
                        c3 = tp1 * t * tm * (1.0f / 6.0f);
            const float ca = (1.0f - Vb) * K1 / a;
            const float al = Vb, be = ca * k3, ga = ca * k2;
            const int b0 = i0 - 1;
            const float4 q0 = qt[b0], q1 = qt[b0 + 1], q2 = qt[b0 + 2], q3 = qt[b0 + 3];
            const float yg = fmaf(c0, q0.x, fmaf(c1, q1.x, fmaf(c2, q2.x, c3 * q3.x)));
            const float cg = fmaf(c0, q0.y, fmaf(c1, q1.y, fmaf(c2, q2.y, c3 * q3.y)));
            const float g0g = fmaf(c0, q0.z, fmaf(c1, q1.z, fmaf(c2, q2.z, c3 * q3.z)));
            const float gg = fmaf(c0, q0.w, fmaf(c1, q1.w, fmaf(c2, q2.w, c3 * q3.w)));
            // d = y.y - 2 y.x + x.x
            const float yx = fmaf(al, yc, fmaf(be, yg0, ga * yg));
            const float xx = fmaf(al * al, cc, fmaf(be * be, g00, fmaf(ga * ga, gg,
                             2.0f * fmaf(al * be, cg0, fmaf(al * ga, cg, be * ga * g0g)))));
            const float d = fmaf(-2.0f, yx, yy) + xx;
            keys[i] = d;
            if (A.u_dump) {
#pragma unroll
                for (int p = 0; p < LA_P; ++p) A.u_dump[((size_t)j * A.M + i) * LA_P + p] = u[p];
            }
            if (A.d_dump) A.d_dump[(size_t)j * A.M + i] = d;
        }
        __syncthreads();

        // ---- the k-th distance K (and the median accepted distance Km)
        uint32_t K = 0, Km = 0;
        int need_ties = 1;
        bool fast = A.n_pilot > 0, have_med = false;
        if (fast) {
            // pivots: 256 bins over the order-preserving integer image of the first n_pilot
            // proposals' keys (an i.i.d. sample), each 2^shift integers wide; lo = the lower
            // edge of the bin holding sample rank r_lo, hi = the upper edge of the bin holding
            // rank r_hi, so lo <= that order statistic <= ... <= hi exactly
            uint32_t* redu = (uint32_t*)red;
            uint32_t kmn = 0xFFFFFFFFu, kmx = 0u;
            for (int i = threadIdx.x; i < A.n_pilot; i += blockDim.x) {
                const uint32_t k = f2key(keys[i]);
                kmn = min(kmn, k);
                kmx = max(kmx, k);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                kmn = min(kmn, __shfl_xor_sync(0xFFFFFFFFu, kmn, o));
                kmx = max(kmx, __shfl_xor_sync(0xFFFFFFFFu, kmx, o));
            }
            if (lane == 0) { redu[wp] = kmn; redu[16 + wp] = kmx; }
            for (int b2 = threadIdx.x; b2 < 512; b2 += blockDim.x) hist[b2] = 0;
            __syncthreads();
            kmn = redu[0];
            kmx = redu[16];
            for (int q = 1; q < nw; ++q) { kmn = min(kmn, redu[q]); kmx = max(kmx, redu[16 + q]); }
            int shift = 0;
            while (((kmx - kmn) >> shift) >= 256u) ++shift;
            for (int i = threadIdx.x; i < A.n_pilot; i += blockDim.x) atomicAdd(&hist[(f2key(keys[i]) - kmn) >> shift], 1u);
            __syncthreads();
            if (wp == 0) warp_find_bin(hist, A.r_lo, lane, &sh[0], &sh[1]);
            if (wp == 1) warp_find_bin(hist, A.r_hi, lane, &sh[2], &sh[3]);
            __syncthreads();
            const uint32_t lo = kmn + ((uint32_t)sh[0] << shift);
            const uint64_t hi64 = (uint64_t)kmn + ((uint64_t)(sh[2] + 1) << shift) - 1u;
            const uint32_t hi = hi64 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)hi64;
            int cl = 0;
            for (int i0 = s0; i0 < s1; i0 += 32) {
                const int i = i0 + lane;
                const float kf = i < s1 ? keys[i] : 0.0f;
                const uint32_t kk = f2key(kf);
                cl += __popc(__ballot_sync(0xFFFFFFFFu, i < s1 && kk < lo));
                const bool in = i < s1 && kk >= lo && kk <= hi;
                const uint32_t bc = __ballot_sync(0xFFFFFFFFu, in);
                if (bc) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(&sh[4], __popc(bc));
                    base = __shfl_sync(0xFFFFFFFFu, base, 0) + __popc(bc & below);
                    if (in && base < LA_CAP) { ckey[base] = kf; cidx[base] = i; }
                }
            }
            if (lane == 0) { wcnt[wp] = cl; wcnt[16 + wp] = 0; }
            for (int b2 = threadIdx.x; b2 < 512; b2 += blockDim.x) hist[b2] = 0;
            __syncthreads();
            const int n_c = sh[4];
            int n_lt = 0;
            for (int q = 0; q < nw; ++q) n_lt += wcnt[q];
            fast = n_lt <= A.k - 1 && n_lt + n_c >= A.k && n_c <= LA_CAP;   // block-uniform
            if (fast) {
                const int rm = (A.k - 1) / 2;
                have_med = rm >= n_lt;
                const int rk0 = A.k - 1 - n_lt, rk1 = have_med ? rm - n_lt : rk0;
                // the candidates' keys lie in [lo, hi]: 256 bins of 2^shift2 integers there,
                // then the members of the bins holding the two ranks, resolved by counting
                int shift2 = 0;
                while (((hi - lo) >> shift2) >= 256u) ++shift2;
                for (int c = threadIdx.x; c < n_c; c += blockDim.x) atomicAdd(&hist[(f2key(ckey[c]) - lo) >> shift2], 1u);
                __syncthreads();
                if (wp == 0) warp_find_bin(hist, rk0, lane, &sh[0], &sh[1]);
                if (wp == 1) warp_find_bin(hist, rk1, lane, &sh[2], &sh[3]);
                __syncthreads();
                const int b0 = sh[0], r0 = sh[1], b1 = sh[2], r1 = sh[3];
                const int m0 = (int)hist[b0], m1 = (int)hist[b1];
                bool small = m0 <= 128 && m1 <= 128;
                if (small) {
                    // gather both bins' members (as integer keys) into the two halves of hist
                    __syncthreads();
                    if (threadIdx.x < 2) sh[5 + threadIdx.x] = 0;
                    __syncthreads();
                    for (int c0 = 0; c0 < n_c; c0 += blockDim.x) {
                        const int c = c0 + threadIdx.x;
                        const uint32_t k = c < n_c ? f2key(ckey[c]) : 0u;
                        const int bin = c < n_c ? (int)((k - lo) >> shift2) : -1;
                        if (bin == b0) hist[atomicAdd(&sh[5], 1)] = k;
                        if (bin == b1 && b1 != b0) hist[256 + atomicAdd(&sh[6], 1)] = k;
                    }
                    __syncthreads();
                    // warp 0: the member of rank r0 in bin b0 (and its rank among equal keys);
                    // warp 1: the member of rank r1 in bin b1
                    if (wp < 2) {
                        const uint32_t* mem = (wp == 1 && b1 != b0) ? hist + 256 : hist;
                        const int m = (wp == 1 && b1 != b0) ? m1 : m0;
                        const int r = wp == 0 ? r0 : r1;
                        uint32_t kv = 0u;
                        int tr = 0;
                        bool got = false;
                        for (int a2 = lane; a2 < m; a2 += 32) {
                            const uint32_t v = mem[a2];
                            int lt = 0, eq = 0;
                            for (int u = 0; u < m; ++u) {
                                lt += mem[u] < v;
                                eq += mem[u] == v;
                            }
                            if (lt <= r && r < lt + eq) { kv = v; tr = r - lt; got = true; }
                        }
                        const uint32_t who = __ballot_sync(0xFFFFFFFFu, got);
                        const int src = who ? __ffs(who) - 1 : 0;
                        kv = __shfl_sync(0xFFFFFFFFu, kv, src);
                        tr = __shfl_sync(0xFFFFFFFFu, tr, src);
                        if (lane == 0) { sh[7 * wp] = (int)kv; if (wp == 0) sh[1] = tr; }
                    }
                    __syncthreads();
                    K = (uint32_t)sh[0];
                    Km = (uint32_t)sh[7];
                    need_ties = sh[1] + 1;     // k minus the number of keys strictly below K
                } else {
                    uint32_t sel[2];
                    int ties[2];
                    block_select2(ckey, n_c, rk0, rk1, hist, sh, sel, ties);
                    K = sel[0];
                    Km = sel[1];
                    need_ties = ties[0] + 1;
                }
                for (int c = threadIdx.x; c < n_c; c += blockDim.x) {
                    const uint32_t kk = f2key(ckey[c]);
                    const int w = cidx[c] / seg;
                    if (kk < K) atomicAdd(&wcnt[w], 1);
                    else if (kk == K) atomicAdd(&wcnt[16 + w], 1);
                }
                __syncthreads();
            }
        }
        if (!fast) {
            uint32_t sel[2];
            int ties[2];
            block_select2(keys, A.M, A.k - 1, (A.k - 1) / 2, hist, sh, sel, ties);
            K = sel[0];
            Km = sel[1];
            have_med = true;
            need_ties = ties[0] + 1;
            int cl = 0, ct = 0;
            for (int i0 = s0; i0 < s1; i0 += 32) {
                const int i = i0 + lane;
                const uint32_t kk = i < s1 ? f2key(keys[i]) : 0u;
                cl += __popc(__ballot_sync(0xFFFFFFFFu, i < s1 && kk < K));
                ct += __popc(__ballot_sync(0xFFFFFFFFu, i < s1 && kk == K));
            }
            if (lane == 0) { wcnt[wp] = cl; wcnt[16 + wp] = ct; }
            __syncthreads();
        }

        // ---- ordered compaction: warp wp places its segment's accepted indices after
        // those of the lower warps, so acc lists the accepted set by increasing index
        {
            int pl0 = 0, pt0 = 0;
            for (int q = 0; q < wp; ++q) { pl0 += wcnt[q]; pt0 += wcnt[16 + q]; }
            for (int i0 = s0; i0 < s1; i0 += 32) {
                const int i = i0 + lane;
                const uint32_t kk = i < s1 ? f2key(keys[i]) : 0u;
                const bool isl = i < s1 && kk < K, ist = i < s1 && kk == K;
                const uint32_t bl = __ballot_sync(0xFFFFFFFFu, isl), bt = __ballot_sync(0xFFFFFFFFu, ist);
                const int pl = pl0 + __popc(bl & below), pt = pt0 + __popc(bt & below);
                if (isl) acc[pl + min(pt, need_ties)] = i;
                else if (ist && pt < need_ties) acc[pl + pt] = i;
                pl0 += __popc(bl);
                pt0 += __popc(bt);
            }
        }
        __syncthreads();
        if (!have_med) {
            // the median lies below the bracket: select it among the k accepted keys
            if (threadIdx.x < A.k) wacc[threadIdx.x] = keys[acc[threadIdx.x]];
            __syncthreads();
            uint32_t sel[2];
            block_select2(wacc, A.k, (A.k - 1) / 2, (A.k - 1) / 2, hist, sh, sel, nullptr);
            Km = sel[0];
        }
        if (threadIdx.x == 0) A.dmed[j] = key2f(Km);
        __syncthreads();

        // weights 1/q, normalised over the accepted set; accepted values
        float lw = -3.0e38f;
        float vals[LA_C] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (threadIdx.x < A.k) {
            float u[LA_P];
            draw_u(A, tp, j, acc[threadIdx.x], u);
            lw = 0.0f;
#pragma unroll
            for (int p = 0; p < LA_P; ++p) {
                lw -= tn_logpdf(tp[p], u[p]);
                vals[p] = A.lo[p] + (A.hi[p] - A.lo[p]) * u[p];
            }
            vals[4] = vals[0] * vals[2] / (vals[1] + vals[2]);
        }
        const float lmax = block_max(lw, red);
        const float wu = threadIdx.x < A.k ? expf(lw - lmax) : 0.0f;
        const float wsum = block_sum(wu, red);
        const float W = wu / wsum;
        const float s2 = block_sum(W * W, red);
        if (threadIdx.x < LA_KMAX) {
            wacc[threadIdx.x] = W;
#pragma unroll
            for (int c = 0; c < LA_C; ++c) sv[c * LA_KMAX + threadIdx.x] = vals[c];
        }
        if (threadIdx.x == 0) {
            A.ess[j] = 1.0f / s2;
            A.ynorm[j] = yy;
        }
        __syncthreads();
        // per column c, warps 2c and 2c + 1: the weighted mean and SD (two passes, per-lane
        // partial sums then a shuffle tree; warp 2c), and the weighted 2.5 % (warp 2c) or
        // 97.5 % (warp 2c + 1) quantile: the smallest accepted value v whose cumulative weight
        // sum_{v_r <= v} W_r reaches the level, found by bisection on the order-preserving
        // integer image of the values
        if (wp < 2 * LA_C) {
            const int c = wp >> 1;
            const bool upper = wp & 1;
            constexpr int PER = LA_KMAX / 32;
            float v[PER], wv[PER];
            uint32_t kv[PER];
            uint32_t kmin = 0xFFFFFFFFu, kmax = 0u;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int r = q * 32 + lane;
                const bool ok = r < A.k;
                v[q] = ok ? sv[c * LA_KMAX + r] : 0.0f;
                wv[q] = ok ? wacc[r] : 0.0f;
                kv[q] = ok ? f2key(v[q]) : 0xFFFFFFFFu;
                if (ok) { kmin = min(kmin, kv[q]); kmax = max(kmax, kv[q]); }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                kmin = min(kmin, __shfl_xor_sync(0xFFFFFFFFu, kmin, o));
                kmax = max(kmax, __shfl_xor_sync(0xFFFFFFFFu, kmax, o));
            }
            const float level = upper ? 0.975f : 0.025f;
            uint32_t lo = kmin, hi = kmax;
            while (lo < hi) {
                const uint32_t mid = lo + ((hi - lo) >> 1);
                float cw = 0.0f;
#pragma unroll
                for (int q = 0; q < PER; ++q) cw += kv[q] <= mid ? wv[q] : 0.0f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cw += __shfl_xor_sync(0xFFFFFFFFu, cw, o);
                if (cw >= level) hi = mid;
                else lo = mid + 1;
            }
            if (upper) {
                if (lane == 0) A.qhi[j * LA_C + c] = key2f(lo);
            } else {
                float m = 0.0f;
#pragma unroll
                for (int q = 0; q < PER; ++q) m = fmaf(wv[q], v[q], m);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xFFFFFFFFu, m, o);
                float v2 = 0.0f;
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    const float e = v[q] - m;
                    v2 = fmaf(wv[q] * e, e, v2);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v2 += __shfl_xor_sync(0xFFFFFFFFu, v2, o);
                if (lane == 0) {
                    A.mean[j * LA_C + c] = m;
                    A.sd[j * LA_C + c] = sqrtf(v2);
                    A.qlo[j * LA_C + c] = key2f(lo);
                }
            }
        }
    }
}

int mlp_dims_ok(int D, int H, int O) {
    VPET_ARG(D >= 1 && D <= 4096 && H >= 1 && H <= 4096 && O >= 1 && O <= 64, "mlp: dimensions out of range");
    return ABC_OK;
}

size_t mlp_params(int D, int H, int O) { return (size_t)H * D + H + (size_t)H * H + H + (size_t)O * H + O; }

// forward pass: z1 = X bf16(W1)^T + b1, z2 = gelu(z1) bf16(W2)^T + b2, out = gelu(z2) bf16(W3)^T + b3
int mlp_forward(const float* prm, int D, int H, int O, const float* X, int64_t B, float* out, float* z1, float* z2,
                cudaStream_t s) {
    const float* W1 = prm;
    const float* b1 = W1 + (size_t)H * D;
    const float* W2 = b1 + H;
    const float* b2 = W2 + (size_t)H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + (size_t)O * H;
    const int Bi = (int)B;
    int rc;
    if ((rc = gemm(GemmArgs{X, D, 1, W1, 1, D, z1, H, b1, Bi, H, D, 0, 0, 1}, s))) return rc;
    if ((rc = gemm(GemmArgs{z1, H, 1, W2, 1, H, z2, H, b2, Bi, H, H, 1, 0, 1}, s))) return rc;
    return gemm(GemmArgs{z2, H, 1, W3, 1, H, out, O, b3, Bi, O, H, 1, 0, 1}, s);
}

}  // namespace

extern "C" int abc_mlp_status(int32_t* timeout_host) {
    vpet::clear_error();
    VPET_ARG(timeout_host, "abc_mlp_status: null pointer");
    int v = 0;
    VPET_CUDA(cudaMemcpyFromSymbol(&v, g_mlp_timeout, sizeof v));
    *timeout_host = v;
    if (v) {
        const int zero = 0;
        VPET_CUDA(cudaMemcpyToSymbol(g_mlp_timeout, &zero, sizeof zero));
    }
    return ABC_OK;
}

extern "C" size_t abc_mlp_param_count(int32_t D, int32_t H, int32_t O) {
    if (D < 1 || H < 1 || O < 1) return 0;
    return mlp_params(D, H, O);
}

extern "C" size_t abc_mlp_workspace_size(int32_t D, int32_t H, int32_t O, int64_t B) {
    if (D < 1 || H < 1 || O < 1 || B < 1) return 0;
    // z1, z2, dh, dz (B x H each), out, dout (B x O each), split-K slabs
    return sizeof(float) * ((size_t)B * H * 4 + (size_t)B * O * 2 + (size_t)GEMM_PART_FLOATS) + 256;
}

extern "C" int abc_mlp_init(uint64_t seed, int32_t D, int32_t H, int32_t O, float* params_dev, void* stream) {
    vpet::clear_error();
    int rc = mlp_dims_ok(D, H, O);
    if (rc) return rc;
    VPET_ARG(params_dev, "abc_mlp_init: null pointer");
    const int64_t n = (int64_t)mlp_params(D, H, O);
    k_mlp_init<<<(unsigned)vpet_ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(params_dev, D, H, O, seed);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

extern "C" int abc_mlp_features(const float* y_dev, int64_t J, int32_t ldy, int32_t L, const float* w_host,
                                float* feat_dev, void* stream) {
    vpet::clear_error();
    VPET_ARG(w_host, "abc_mlp_features: null weights");
    VPET_ARG(L >= 1 && L <= MAXL && ldy >= L && J >= 0, "abc_mlp_features: bad sizes");
    VPET_ARG(J == 0 || (y_dev && feat_dev), "abc_mlp_features: null pointer");
    if (J == 0) return ABC_OK;
    FrameW W;
    memset(&W, 0, sizeof W);
    for (int l = 0; l < L; ++l) W.w[l] = w_host[l];
    k_features<<<(unsigned)vpet_ceil_div(J, 8), 256, 0, (cudaStream_t)stream>>>(y_dev, J, ldy, L, W, feat_dev);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

extern "C" int abc_mlp_forward(const float* params_dev, int32_t D, int32_t H, int32_t O, const float* X_dev,
                               int64_t B, float* out_dev, void* work_dev, size_t work_bytes, void* stream) {
    vpet::clear_error();
    int rc = mlp_dims_ok(D, H, O);
    if (rc) return rc;
    VPET_ARG(B >= 1 && B < (1 << 30), "abc_mlp_forward: batch must be in [1, 2^30)");
    VPET_ARG(params_dev && X_dev && out_dev && work_dev, "abc_mlp_forward: null pointer");
    if (work_bytes < abc_mlp_workspace_size(D, H, O, B)) {
        vpet::set_error("abc_mlp_forward: workspace too small");
        return ABC_ERR_WORKSPACE;
    }
    float* z1 = (float*)work_dev;
    float* z2 = z1 + (size_t)B * H;
    return mlp_forward(params_dev, D, H, O, X_dev, B, out_dev, z1, z2, (cudaStream_t)stream);
}

extern "C" int abc_mlp_loss_grad(const float* params_dev, int32_t D, int32_t H, int32_t P, const float* X_dev,
                                 const float* T_dev, int64_t B, void* work_dev, size_t work_bytes, float* grad_dev,
                                 float* loss_dev, void* stream) {
    vpet::clear_error();
    VPET_ARG(P >= 1 && P <= 32, "abc_mlp_loss_grad: P must be in [1, 32]");
    const int O = 2 * P;
    int rc = mlp_dims_ok(D, H, O);
    if (rc) return rc;
    VPET_ARG(B >= 1 && B < (1 << 30), "abc_mlp_loss_grad: batch must be in [1, 2^30)");
    VPET_ARG(params_dev && X_dev && T_dev && grad_dev && loss_dev && work_dev, "abc_mlp_loss_grad: null pointer");
    if (work_bytes < abc_mlp_workspace_size(D, H, O, B)) {
        vpet::set_error("abc_mlp_loss_grad: workspace too small");
        return ABC_ERR_WORKSPACE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    float* z1 = (float*)work_dev;
    float* z2 = z1 + (size_t)B * H;
    float* dh = z2 + (size_t)B * H;
    float* dz = dh + (size_t)B * H;
    float* out = dz + (size_t)B * H;
    float* dout = out + (size_t)B * O;
    float* part = dout + (size_t)B * O;
    if ((rc = mlp_forward(params_dev, D, H, O, X_dev, B, out, z1, z2, s))) return rc;
    VPET_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(float), s));
    k_trunc_nll<<<(unsigned)vpet_ceil_div(B * P, 256), 256, 0, s>>>(out, T_dev, (int)B, P, dout, loss_dev);
    VPET_LAUNCH_CHECK();
    const float* W2 = params_dev + (size_t)H * D + H;
    const float* W3 = W2 + (size_t)H * H + H;
    float* gW1 = grad_dev;
    float* gb1 = gW1 + (size_t)H * D;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + (size_t)H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + (size_t)O * H;
    const int Bi = (int)B;
    // layer 3: gW3 = dout^T gelu(z2), gb3 = colsum(dout), dh = dout bf16(W3)
    if ((rc = gemm(GemmArgs{dout, 1, O, z2, H, 1, gW3, H, nullptr, O, H, Bi, 0, 1, 0, part, GEMM_PART_FLOATS}, s))) return rc;
    k_colsum<<<(unsigned)vpet_ceil_div(O, 32), 256, 0, s>>>(dout, Bi, O, gb3);
    VPET_LAUNCH_CHECK();
    if ((rc = gemm(GemmArgs{dout, O, 1, W3, H, 1, dh, H, nullptr, Bi, H, O, 0, 0, 1}, s))) return rc;
    // layer 2: dz = dh gelu'(z2), gW2 = dz^T gelu(z1), gb2 = colsum(dz), dh = dz bf16(W2)
    k_gelu_back<<<(unsigned)vpet_ceil_div(B * H, 256), 256, 0, s>>>(dh, z2, dz, B * H);
    VPET_LAUNCH_CHECK();
    if ((rc = gemm(GemmArgs{dz, 1, H, z1, H, 1, gW2, H, nullptr, H, H, Bi, 0, 1, 0, part, GEMM_PART_FLOATS}, s))) return rc;
    k_colsum<<<(unsigned)vpet_ceil_div(H, 32), 256, 0, s>>>(dz, Bi, H, gb2);
    VPET_LAUNCH_CHECK();
    if ((rc = gemm(GemmArgs{dz, H, 1, W2, H, 1, dh, H, nullptr, Bi, H, H, 0, 0, 1}, s))) return rc;
    // layer 1: dz = dh gelu'(z1), gW1 = dz^T X, gb1 = colsum(dz)
    k_gelu_back<<<(unsigned)vpet_ceil_div(B * H, 256), 256, 0, s>>>(dh, z1, dz, B * H);
    VPET_LAUNCH_CHECK();
    if ((rc = gemm(GemmArgs{dz, 1, H, X_dev, D, 1, gW1, D, nullptr, H, D, Bi, 0, 0, 0, part, GEMM_PART_FLOATS}, s))) return rc;
    k_colsum<<<(unsigned)vpet_ceil_div(H, 32), 256, 0, s>>>(dz, Bi, H, gb1);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

extern "C" int abc_unit_box(const float* theta_dev, int64_t N, int32_t ldtheta, int32_t P, const double* lo_host,
                            const double* hi_host, float* t_dev, void* stream) {
    vpet::clear_error();
    VPET_ARG(lo_host && hi_host, "abc_unit_box: null bounds");
    VPET_ARG(P >= 1 && P <= 8 && ldtheta >= P && N >= 0, "abc_unit_box: bad sizes");
    VPET_ARG(N == 0 || (theta_dev && t_dev), "abc_unit_box: null pointer");
    Box b;
    memset(&b, 0, sizeof b);
    for (int p = 0; p < P; ++p) {
        VPET_ARG(hi_host[p] > lo_host[p], "abc_unit_box: need lo < hi");
        b.lo[p] = (float)lo_host[p];
        b.inv[p] = (float)(1.0 / (hi_host[p] - lo_host[p]));
    }
    if (N == 0) return ABC_OK;
    k_unit_box<<<(unsigned)vpet_ceil_div(N * P, 256), 256, 0, (cudaStream_t)stream>>>(theta_dev, N, ldtheta, P, b,
                                                                                     t_dev);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

extern "C" int abc_adam_update(float* params_dev, const float* grad_dev, float* m_dev, float* v_dev, int64_t n,
                               float lr, float beta1, float beta2, float eps, int32_t t, void* stream) {
    vpet::clear_error();
    VPET_ARG(params_dev && grad_dev && m_dev && v_dev, "abc_adam_update: null pointer");
    VPET_ARG(n >= 1 && t >= 1 && beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f,
             "abc_adam_update: bad arguments");
    const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
    k_adam<<<(unsigned)vpet_ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(params_dev, grad_dev, m_dev, v_dev, n,
                                                                              lr, beta1, beta2, eps, c1, c2);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

extern "C" int abc_add_noise(const float* x_dev, int64_t N, int32_t ldx, const abc_frames* frames, double half_life,
                             double q_lo, double q_hi, uint64_t seed, int64_t first_index, float* y_dev, int32_t ldy,
                             void* stream) {
    vpet::clear_error();
    VPET_ARG(frames && frames->t_start && frames->t_end, "abc_add_noise: null frames");
    VPET_ARG(frames->L >= 1 && frames->L <= MAXL && ldx >= frames->L && ldy >= frames->L, "abc_add_noise: bad sizes");
    VPET_ARG(half_life > 0 && q_lo >= 0 && q_hi >= q_lo, "abc_add_noise: bad noise parameters");
    VPET_ARG(N >= 0 && (N == 0 || (x_dev && y_dev)), "abc_add_noise: null pointer");
    NoiseFrames F;
    memset(&F, 0, sizeof F);
    F.L = frames->L;
    for (int l = 0; l < F.L; ++l) {
        F.tmid[l] = (float)(0.5 * (frames->t_start[l] + frames->t_end[l]));
        F.dt[l] = (float)(frames->t_end[l] - frames->t_start[l]);
        VPET_ARG(F.dt[l] > 0.0f, "abc_add_noise: empty frame");
    }
    if (N == 0) return ABC_OK;
    k_add_noise<<<(unsigned)vpet_ceil_div(N, 8), 256, 0, (cudaStream_t)stream>>>(
        x_dev, N, ldx, F, (float)(0.69314718055994531 / half_life), (float)q_lo, (float)q_hi, seed, first_index,
        y_dev, ldy);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

extern "C" size_t abc_local_abc_smem_bytes(int32_t T, int32_t L, int32_t M) {
    if (T < 1 || L < 1 || M < 1) return 0;
    const size_t kreg = (size_t)M > (size_t)LA_C * LA_KMAX ? (size_t)M : (size_t)LA_C * LA_KMAX;
    // qt (4 T), cps + ys, keys, acc + wacc, red, 2 histograms, sh, warp counts, scal, candidates
    return sizeof(float) * (4 * (size_t)T + 2 * MAXL + kreg + 2 * LA_KMAX + 64 + 512 + 8 + 32 + 8 + 2 * LA_CAP);
}

__global__ void k_table_frame_major(const float* __restrict__ rows, int T, int L, int ld, float* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= T * L) return;
    const int l = e / T, i = e - l * T;
    out[e] = rows[(size_t)i * ld + l];
}

extern "C" int abc_local_abc_table(const float* rows_dev, int32_t T, int32_t L, int32_t ld, float* table_dev,
                                   void* stream) {
    vpet::clear_error();
    VPET_ARG(T >= 1 && L >= 1 && L <= MAXL && ld >= L && (int64_t)T * L < (1LL << 31),
             "abc_local_abc_table: bad sizes");
    VPET_ARG(rows_dev && table_dev, "abc_local_abc_table: null pointer");
    k_table_frame_major<<<(unsigned)vpet_ceil_div((int64_t)T * L, 256), 256, 0, (cudaStream_t)stream>>>(
        rows_dev, T, L, ld, table_dev);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}

extern "C" int abc_local_abc(const float* y_dev, int64_t J, int32_t ldy, int32_t L, const float* w_host,
                             const float* prop_dev, const float* table_dev, int32_t T, double a_max,
                             const float* cp_frames_dev, const double* lo_host, const double* hi_host, int32_t M,
                             int32_t k, float sigma_scale, uint64_t seed, float* mean_dev, float* sd_dev, float* qlo_dev, float* qhi_dev,
                             float* ess_dev, float* dmed_dev, float* ynorm_dev, float* u_dump_dev, float* d_dump_dev,
                             void* stream) {
    vpet::clear_error();
    VPET_ARG(w_host && lo_host && hi_host, "abc_local_abc: null host pointer");
    VPET_ARG(L >= 1 && L <= MAXL && ldy >= L && J >= 0 && T >= 8 && a_max > 0, "abc_local_abc: bad sizes");
    VPET_ARG(k >= 1 && k <= LA_KMAX && M >= k && M <= (1 << 20), "abc_local_abc: need 1 <= k <= 256 and k <= M");
    VPET_ARG(sigma_scale > 0.0f && sigma_scale <= 100.0f, "abc_local_abc: sigma_scale must be in (0, 100]");
    for (int p = 0; p < LA_P; ++p)
        VPET_ARG(lo_host[p] <= hi_host[p] && lo_host[p] >= 0.0, "abc_local_abc: prior box must satisfy 0 <= lo <= hi");
    VPET_ARG(lo_host[1] + lo_host[2] > 0.0 && hi_host[1] + hi_host[2] <= a_max,
             "abc_local_abc: k2 + k3 must stay in (0, a_max]");
    const size_t smem = abc_local_abc_smem_bytes(T, L, M);
    VPET_ARG(smem <= 227 * 1024, "abc_local_abc: T tabulated products and M distances exceed 227 KB of shared memory");
    if (J == 0) return ABC_OK;
    VPET_ARG(y_dev && prop_dev && table_dev && cp_frames_dev, "abc_local_abc: null device input");
    VPET_ARG(mean_dev && sd_dev && qlo_dev && qhi_dev && ess_dev && dmed_dev && ynorm_dev,
             "abc_local_abc: null output");
    LocalArgs A;
    memset(&A, 0, sizeof A);
    A.y = y_dev;
    A.J = J;
    A.ldy = ldy;
    A.L = L;
    for (int l = 0; l < L; ++l) A.w[l] = w_host[l];
    A.prop = prop_dev;
    A.table = table_dev;
    A.cpf = cp_frames_dev;
    A.T = T;
    // Bracketing of the k-th distance by a pilot sample: pivots at the sample ranks
    // 4 standard deviations (plus one) either side of where the k-th of M falls; used
    // when the keys expected below the lower pivot leave room for the median and the
    // expected candidates fit the buffer with a factor 2 to spare.
    if (M >= 2048) {
        const int n = M < LA_PILOT ? M : LA_PILOT;
        const double pq = (k - 0.5) / M, mu = n * pq, sd = sqrt(n * pq * (1.0 - pq)) + 1.0;
        const int rl = (int)floor(mu - 4.0 * sd) - 1, rh = (int)ceil(mu + 4.0 * sd) + 1;
        const int r_lo = rl < 0 ? 0 : rl, r_hi = rh > n - 1 ? n - 1 : rh;
        const double below = (r_lo + 1.0) * M / (n + 1.0), cand = (r_hi - r_lo + 1.0) * M / (n + 1.0);
        if (below <= 0.5 * (k - 1) && cand <= 0.5 * LA_CAP) {
            A.n_pilot = n;
            A.r_lo = r_lo;
            A.r_hi = r_hi;
        }
    }
    A.a_max = (float)a_max;
    for (int p = 0; p < LA_P; ++p) {
        A.lo[p] = (float)lo_host[p];
        A.hi[p] = (float)hi_host[p];
    }
    A.M = M;
    A.k = k;
    A.sigma_scale = sigma_scale;
    A.seed = seed;
    A.mean = mean_dev;
    A.sd = sd_dev;
    A.qlo = qlo_dev;
    A.qhi = qhi_dev;
    A.ess = ess_dev;
    A.dmed = dmed_dev;
    A.ynorm = ynorm_dev;
    A.u_dump = u_dump_dev;
    A.d_dump = d_dump_dev;
    VPET_CUDA(cudaFuncSetAttribute(k_local_abc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    VPET_CUDA(cudaGetDevice(&dev));
    VPET_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    VPET_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_local_abc, LA_THREADS, smem));
    VPET_ARG(per_sm >= 1, "abc_local_abc: kernel does not fit on an SM with this shared memory");
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > J) grid = J;
    k_local_abc<<<(unsigned)grid, LA_THREADS, smem, (cudaStream_t)stream>>>(A);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}
