// Simulated frame-mean TACs (Algorithm 1, step 3), one thread per prior draw.
//
// Every measured curve here is a sum of convolutions of exponentials:
//   2TCM (Eq. 1-2):  C_t = Vb C_p + (1 - Vb) [A1 e^{-a1 t} + A2 e^{-a2 t}] (*) C_p
//   MRTM (Eq. 3, gamma = 0):  C_t = R1 C_r + (k2 - R1 k2a) e^{-k2a t} (*) C_r
// and each input term t^m e^{-c t} is m! times the m+1-fold self-convolution of
// e^{-c t}.  So C_t is a weighted sum of "chains"  Conv(x_0..x_n)(t) =
// (e^{-x_0 t} (*) ... (*) e^{-x_n t})(t), which equals (-1)^n times the divided
// difference of f(x) = e^{-x t} over the nodes x_0..x_n.
//
// Numerics (fp32 throughout):
//  * Conv over sorted nodes is built bottom-up over node ranges: a range whose
//    spread times t exceeds 1 uses the divided-difference recursion (no
//    catastrophic cancellation at that spread); a narrower range uses the
//    Taylor series in the node offsets, which is exact in the limit of equal
//    rates.  Near-degenerate rates (k2 + k3 close to an input rate) therefore
//    need no fp64 and no special case.
//  * Frame integrals avoid the difference F(t_e) - F(t_s) of running integrals.
//    With s = t - t_s,  Conv(x_0..x_n)(t_s + s) = sum_r Conv(x_0..x_r)(t_s) Conv(x_r..x_n)(s)
//    (the semigroup property of the convolution), so
//    int_{t_s}^{t_e} Conv = sum_r Conv(x_0..x_r)(t_s) * Conv(0, x_r..x_n)(dt):
//    a sum of positive products.  The dt-dependent factors are computed once
//    per run of equal-duration frames.
//  * lp-ntPET (Eq. 3-4) has no closed form once the activation starts: it is
//    MRTM up to t_D, then Z = C_t - R1 C_r obeys Z' = (k2 - R1 a(t)) C_r - a(t) Z
//    with a = k2a + gamma g(t), integrated by an exponential integrator (a frozen
//    at its Simpson average over each step, the forcing linear across the step),
//    exact phi-function weights for both Z and its frame integral.
#include <string.h>

#include "common.cuh"

#define SIM_MAXL 64
#define SIM_MAXT 16
#define SIM_THREADS 128

namespace {

struct SimParams {
    int L;
    int nseg;
    float ts[SIM_MAXL];
    float dt[SIM_MAXL];
    int seg_begin[SIM_MAXL + 1];   // runs of consecutive frames with the same duration
    int nterms;
    float c[SIM_MAXT];
    float a[SIM_MAXT][3];          // coefficient of Conv(c^(m+1)), i.e. a_m * m!
    float lp_h;                    // lp-ntPET integrator step (min)
    int lp_ntab;                   // lp-ntPET: C_r tabulated at t = i lp_h, i < lp_ntab (0: none)
};

constexpr int SIM_MAX_TAB = 4096;

// 1/n! for n = 0..19 (folds to a constant wherever n is known at compile time).
__host__ __device__ __forceinline__ float inv_fact(int n) {
    switch (n) {
        case 0: return 1.0f;
        case 1: return 1.0f;
        case 2: return 0.5f;
        case 3: return 1.0f / 6.0f;
        case 4: return 1.0f / 24.0f;
        case 5: return 1.0f / 120.0f;
        case 6: return 1.0f / 720.0f;
        case 7: return 1.0f / 5040.0f;
        case 8: return 1.0f / 40320.0f;
        case 9: return 1.0f / 362880.0f;
        case 10: return 1.0f / 3628800.0f;
        case 11: return 1.0f / 39916800.0f;
        case 12: return 1.0f / 479001600.0f;
        case 13: return 1.0f / 6227020800.0f;
        case 14: return 1.0f / 87178291200.0f;
        case 15: return 1.0f / 1307674368000.0f;
        case 16: return 1.0f / 20922789888000.0f;
        case 17: return 1.0f / 355687428096000.0f;
        case 18: return 1.0f / 6402373705728000.0f;
        default: return 1.0f / 121645100408832000.0f;
    }
}

constexpr int kTaylorTerms = 10;

// Conv over nodes x[i..i+M] (x[i] the smallest) at time t by the Taylor series
// sum_q (-1)^q h_q(u) / (M+q)!  * t^M e^{-x_i t},  u_k = (x_k - x_i) t <= 1,
// h_q the complete homogeneous symmetric polynomial.
template <int N>
__host__ __device__ __forceinline__ float taylor_conv(const float (&x)[N], int i, int M, float t, float e_i) {
    float H[kTaylorTerms + 1];
    H[0] = 1.0f;
#pragma unroll
    for (int q = 1; q <= kTaylorTerms; ++q) H[q] = 0.0f;
#pragma unroll
    for (int k = 1; k < N; ++k) {
        if (k <= M) {
            const float u = (x[i + k] - x[i]) * t;
#pragma unroll
            for (int q = 1; q <= kTaylorTerms; ++q) H[q] = fmaf(u, H[q - 1], H[q]);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int q = kTaylorTerms; q >= 0; --q) s += ((q & 1) ? -H[q] : H[q]) * inv_fact(M + q);
    float tm = 1.0f;
#pragma unroll
    for (int k = 1; k < N; ++k)
        if (k <= M) tm *= t;
    return e_i * tm * s;
}

// V[i][j] = Conv(x_i..x_j)(t) for all ranges of the sorted nodes x[0..N).
template <int N>
__host__ __device__ __forceinline__ void dd_table(const float (&x)[N], float t, float (&V)[N][N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) V[i][i] = expf(-x[i] * t);
#pragma unroll
    for (int len = 2; len <= N; ++len) {
#pragma unroll
        for (int i = 0; i + len - 1 < N; ++i) {
            const int j = i + len - 1;
            const float sp = x[j] - x[i];
            if (sp * t > 1.0f)
                V[i][j] = (V[i][j - 1] - V[i + 1][j]) / sp;
            else
                V[i][j] = taylor_conv<N>(x, i, len - 1, t, V[i][i]);
        }
    }
}

template <int N>
__host__ __device__ __forceinline__ float conv_full(const float (&x)[N], float t) {
    float V[N][N];
    dd_table<N>(x, t, V);
    return V[0][N - 1];
}

// Suffix factors S_r = Conv(0, x_r..x_{N-1})(d), r = 0..N-1.
template <int N, int R>
struct Suffix {
    static __host__ __device__ __forceinline__ void run(const float (&x)[N], float d, float (&S)[N]) {
        float y[N - R + 1];
        y[0] = 0.0f;
#pragma unroll
        for (int k = R; k < N; ++k) y[k - R + 1] = x[k];
        S[R] = conv_full<N - R + 1>(y, d);
        Suffix<N, R + 1>::run(x, d, S);
    }
};
template <int N>
struct Suffix<N, N> {
    static __host__ __device__ __forceinline__ void run(const float (&)[N], float, float (&)[N]) {}
};

template <int N>
__host__ __device__ __forceinline__ void suffix_factors(const float (&x)[N], float d, float (&S)[N]) {
    Suffix<N, 0>::run(x, d, S);
}

// Adds coef * int over each frame [l0, l1) of Conv(x) into acc[l] (frame integrals,
// not yet divided by the duration d).
template <int N>
__host__ __device__ __forceinline__ void accumulate_chain(const float (&x)[N], float coef, const SimParams& p, int l0,
                                                 int l1, float d, float* acc) {
    float S[N];
    suffix_factors<N>(x, d, S);
    for (int l = l0; l < l1; ++l) {
        float V[N][N];
        dd_table<N>(x, p.ts[l], V);
        float s = 0.0f;
#pragma unroll
        for (int r = 0; r < N; ++r) s = fmaf(V[0][r], S[r], s);
        acc[l * SIM_THREADS] += coef * s;
    }
}

// Chain = optional rate `a` (has_a) followed by (m+1) copies of the input rate c.
__host__ __device__ __forceinline__ void chain_dispatch(bool has_a, float a, float c, int m, float coef, const SimParams& p,
                                               int l0, int l1, float d, float* acc) {
    const int n = (has_a ? 1 : 0) + m + 1;
    const bool a_first = has_a && a <= c;
    // sorted nodes
    float x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = c;
    if (has_a) {
        if (a_first) x[0] = a;
        else x[n - 1] = a;
    }
    switch (n) {
        case 1: { float y[1] = {x[0]}; accumulate_chain<1>(y, coef, p, l0, l1, d, acc); break; }
        case 2: { float y[2] = {x[0], x[1]}; accumulate_chain<2>(y, coef, p, l0, l1, d, acc); break; }
        case 3: { float y[3] = {x[0], x[1], x[2]}; accumulate_chain<3>(y, coef, p, l0, l1, d, acc); break; }
        default: { float y[4] = {x[0], x[1], x[2], x[3]}; accumulate_chain<4>(y, coef, p, l0, l1, d, acc); break; }
    }
}

// Closed-form frame integrals of  direct * input + sum_q irf_coef[q] e^{-irf_rate[q] t} (*) input
// for frames in [lbeg, lend), accumulated into acc (stride SIM_THREADS).
// With d_override > 0 the frames [lbeg, lend) are integrated over [ts, ts + d_override).
__host__ __device__ void closed_form_frames(const SimParams& p, float direct, int nirf, const float* irf_coef,
                                   const float* irf_rate, int lbeg, int lend, float* acc, float d_override = 0.0f) {
    const int nseg = d_override > 0.0f ? 1 : p.nseg;
    for (int sg = 0; sg < nseg; ++sg) {
        const int l0 = d_override > 0.0f ? lbeg : max(p.seg_begin[sg], lbeg);
        const int l1 = d_override > 0.0f ? lend : min(p.seg_begin[sg + 1], lend);
        if (l0 >= l1) continue;
        const float d = d_override > 0.0f ? d_override : p.dt[l0];
        for (int i = 0; i < p.nterms; ++i) {
            for (int m = 0; m < 3; ++m) {
                const float am = p.a[i][m];
                if (am == 0.0f) continue;
                if (direct != 0.0f) chain_dispatch(false, 0.0f, p.c[i], m, direct * am, p, l0, l1, d, acc);
                for (int q = 0; q < nirf; ++q)
                    if (irf_coef[q] != 0.0f) chain_dispatch(true, irf_rate[q], p.c[i], m, irf_coef[q] * am, p, l0, l1, d, acc);
            }
        }
    }
}

// ---------------------------------------------------------------- lp-ntPET pieces
// sum over input terms of coef * Conv(rate, c^(m+1)) at time t (pointwise).
__host__ __device__ float conv_rate_input_at(const SimParams& p, float rate, float t) {
    float s = 0.0f;
    for (int i = 0; i < p.nterms; ++i) {
        for (int m = 0; m < 3; ++m) {
            const float am = p.a[i][m];
            if (am == 0.0f) continue;
            const float c = p.c[i];
            const bool a_first = rate <= c;
            float v;
            if (m == 0) {
                float y[2] = {a_first ? rate : c, a_first ? c : rate};
                v = conv_full<2>(y, t);
            } else if (m == 1) {
                float y[3] = {a_first ? rate : c, c, a_first ? c : rate};
                v = conv_full<3>(y, t);
            } else {
                float y[4] = {a_first ? rate : c, c, c, a_first ? c : rate};
                v = conv_full<4>(y, t);
            }
            s = fmaf(am, v, s);
        }
    }
    return s;
}

// Input curve value at t.
__host__ __device__ float input_at(const SimParams& p, float t) {
    float s = 0.0f;
    for (int i = 0; i < p.nterms; ++i) {
        const float e = expf(-p.c[i] * t);
        const float poly = fmaf(fmaf(0.5f * p.a[i][2], t, p.a[i][1]), t, p.a[i][0]);   // a stores a_m * m!
        s = fmaf(poly, e, s);
    }
    return s;
}

// phi_k(-z) = sum_j (-z)^j / (j + k)!  for k = 1, 2, 3 (|z| <= 1 by construction of the step).
__host__ __device__ __forceinline__ void phis(float z, float& p1, float& p2, float& p3) {
    if (z > 0.5f) {
        const float em = expm1f(-z);           // e^{-z} - 1
        p1 = -em / z;
        p2 = (em + z) / (z * z);
        p3 = -(em + z - 0.5f * z * z) / (z * z * z);
        return;
    }
    float a1 = 0.0f, a2 = 0.0f, a3 = 0.0f, pw = 1.0f;
    if (z <= 0.125f) {
        // |z|^6 / 7! < 1e-9: six terms reach fp32 rounding
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            a1 = fmaf(pw, inv_fact(j + 1), a1);
            a2 = fmaf(pw, inv_fact(j + 2), a2);
            a3 = fmaf(pw, inv_fact(j + 3), a3);
            pw *= -z;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            a1 = fmaf(pw, inv_fact(j + 1), a1);
            a2 = fmaf(pw, inv_fact(j + 2), a2);
            a3 = fmaf(pw, inv_fact(j + 3), a3);
            pw *= -z;
        }
    }
    p1 = a1; p2 = a2; p3 = a3;
}

// On the device through the hardware approximations of exp and log (__expf, __logf): their
// relative error, a few 2^-22 here, stays two orders below the integrator's own error
// (the frame means are checked against the FP64 oracle within 1e-4 of the TAC peak).
__host__ __device__ __forceinline__ float gamma_variate(float t, float tD, float inv_tp, float alpha) {
    if (t <= tD) return 0.0f;
    const float x = (t - tD) * inv_tp;      // inv_tp = 1 / (t_P - t_D)
#ifdef __CUDA_ARCH__
    return __expf(alpha * (__logf(x) + 1.0f - x));
#else
    return expf(alpha * (logf(x) + 1.0f - x));
#endif
}

// ---------------------------------------------------------------- kernel
// Frame means of one draw: acc[l * SIM_THREADS] receives x_l (acc zeroed by the caller).
// crtab: C_r at t = i lp_h for i < p.lp_ntab (lp-ntPET; null: evaluate every step).
template <int MODEL>
__host__ __device__ void simulate_draw(const SimParams& p, const float* th, float* acc, const float* crtab = nullptr) {
    if (MODEL == ABC_2TCM_IRR || MODEL == ABC_2TCM_REV) {
        const float K1 = th[0], k2 = th[1], k3 = th[2];
        const float k4 = MODEL == ABC_2TCM_REV ? th[3] : 0.0f;
        const float Vb = MODEL == ABC_2TCM_REV ? th[4] : th[3];
        // impulse response h = A1 e^{-a1 t} + A2 e^{-a2 t} of Eq. 1, both A >= 0
        const float s = k2 + k3 + k4;
        const float u = k2 - k3 - k4;
        const float D = sqrtf(fmaf(u, u, 4.0f * k2 * k3));      // = a2 - a1
        const float a1 = 2.0f * k2 * k4 / (s + D);
        const float a2 = 0.5f * (s + D);
        const float g2 = u >= 0.0f ? 0.5f * (u + D) : 2.0f * k2 * k3 / (D - u);   // a2 - k3 - k4
        const float A1 = D > 0.0f ? K1 * (k3 + k4 - a1) / D : 0.0f;
        const float A2 = D > 0.0f ? K1 * g2 / D : K1;
        const float coef[2] = {(1.0f - Vb) * A1, (1.0f - Vb) * A2};
        const float rate[2] = {a1, a2};
        closed_form_frames(p, Vb, 2, coef, rate, 0, p.L, acc);
    } else {
        const float R1 = th[0], k2 = th[1], k2a = th[1] / (1.0f + th[2]);
        const float B = k2 - R1 * k2a;
        if (MODEL == ABC_MRTM) {
            closed_form_frames(p, R1, 1, &B, &k2a, 0, p.L, acc);
        } else {
            const float gam = th[3], tD = th[4], tPmD = th[5], alpha = th[6];
            // R1 * C_r over every frame, closed form
            closed_form_frames(p, R1, 0, nullptr, nullptr, 0, p.L, acc);
            // Z = B e^{-k2a t} (*) C_r in closed form for frames ending by t_D
            int lsplit = 0;
            while (lsplit < p.L && p.ts[lsplit] + p.dt[lsplit] <= tD) ++lsplit;
            const float zero = 0.0f;
            closed_form_frames(p, zero, 1, &B, &k2a, 0, lsplit, acc);
            // the frame holding t_D: closed form over [ts, tD)
            float t = tD;
            float Z = B * conv_rate_input_at(p, k2a, tD);
            if (lsplit < p.L && p.ts[lsplit] < tD)
                closed_form_frames(p, zero, 1, &B, &k2a, lsplit, lsplit + 1, acc, tD - p.ts[lsplit]);
            // Exponential integrator from t_D to the end.  Steps grow geometrically from
            // t_D (h = t - t_D, at least lp_h / 4096) up to lp_h, which resolves the
            // x^alpha onset of the gamma variate.
            float cr0 = input_at(p, t);
            const float inv_tp = 1.0f / tPmD;
            float g0 = gamma_variate(t, tD, inv_tp, alpha);
            for (int l = lsplit; l < p.L; ++l) {
                const float ts_l = p.ts[l], te = p.ts[l] + p.dt[l];
                float integ = 0.0f;
                int guard = 0;
                while (t < te && guard++ < 100000) {
                    const float stop = t < ts_l ? ts_l : te;     // land exactly on frame edges (gaps allowed)
                    const float h = fminf(fminf(stop - t, p.lp_h), fmaxf(t - tD, p.lp_h * (1.0f / 4096.0f)));
                    // a(t) averaged over the step by Simpson's rule; forcing b = (k2 - R1 a) C_r linear
                    const float gm = gamma_variate(t + 0.5f * h, tD, inv_tp, alpha);
                    const float g1 = gamma_variate(t + h, tD, inv_tp, alpha);
                    const float abar = k2a + gam * (g0 + 4.0f * gm + g1) * (1.0f / 6.0f);
                    // C_r at the step's end: from the table when that end lies on the lp_h grid
                    // (every step between frame edges that are themselves on it), the same
                    // function of the same fp32 time otherwise
                    const float t1 = t + h;
                    const float qf = t1 / p.lp_h;
                    const int qi = (int)qf;
                    const float cr1 = (crtab && (float)qi == qf && qi < p.lp_ntab && (float)qi * p.lp_h == t1)
                                          ? crtab[qi] : input_at(p, t1);
                    const float b0 = (k2 - R1 * (k2a + gam * g0)) * cr0;
                    const float b1 = (k2 - R1 * (k2a + gam * g1)) * cr1;
                    float p1, p2, p3;
                    phis(abar * h, p1, p2, p3);
                    // int_0^h Z = Z0 h phi1 + h^2 (b0 phi2 + (b1 - b0) phi3)
                    if (t >= ts_l) integ += h * fmaf(Z, p1, h * fmaf(b1 - b0, p3, b0 * p2));
                    // Z(h) = e^{-abar h} Z0 + h (b0 phi1 + (b1 - b0) phi2), e^{-z} = 1 - z phi1(z)
                    Z = fmaf(-abar * h, p1, 1.0f) * Z + h * fmaf(b1 - b0, p2, b0 * p1);
                    cr0 = cr1;
                    g0 = g1;
                    t += h;
                }
                acc[l * SIM_THREADS] += integ;
            }
        }
    }
    for (int l = 0; l < p.L; ++l) acc[l * SIM_THREADS] /= p.dt[l];
}

template <int MODEL>
__global__ void __launch_bounds__(SIM_THREADS) k_simulate(SimParams p, const float* __restrict__ theta, int64_t N,
                                                         int ldt, float* __restrict__ x, int ldx) {
    extern __shared__ float s_acc[];   // [L][SIM_THREADS]: frame integrals of this block's draws
    const int tid = threadIdx.x;
    const int64_t n0 = (int64_t)blockIdx.x * SIM_THREADS;
    int slot = tid;                    // the block's draw this thread simulates
    if (MODEL == ABC_LPNTPET) {
        // threads take the block's draws in order of t_D (the integrator runs from t_D to
        // the last frame, so a warp's lanes then take similar numbers of steps); ranks by
        // (order-preserving bits of t_D, position) are a permutation for any values
        __shared__ uint32_t s_key[SIM_THREADS];
        __shared__ int s_slot[SIM_THREADS];
        uint32_t key = 0xFFFFFFFFu;
        if (n0 + tid < N) {
            const uint32_t b = __float_as_uint(theta[(n0 + tid) * ldt + 4]);
            key = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
        }
        s_key[tid] = key;
        __syncthreads();
        int rank = 0;
        for (int i = 0; i < SIM_THREADS; ++i) {
            const uint32_t o = s_key[i];
            rank += (o < key) || (o == key && i < tid);
        }
        s_slot[rank] = tid;
        __syncthreads();
        slot = s_slot[tid];
    }
    const int64_t n = n0 + slot;
    float* acc = s_acc + slot;
    for (int l = 0; l < p.L; ++l) acc[l * SIM_THREADS] = 0.0f;
    float* crtab = nullptr;
    if (MODEL == ABC_LPNTPET && p.lp_ntab > 0) {
        crtab = s_acc + p.L * SIM_THREADS;
        for (int i = tid; i < p.lp_ntab; i += SIM_THREADS) crtab[i] = input_at(p, (float)i * p.lp_h);
        __syncthreads();
    }
    if (n < N) {
        simulate_draw<MODEL>(p, theta + n * ldt, acc, crtab);
    }
    __syncthreads();
    // coalesced write-out of the block's rows
    const int rows = (N - n0) < SIM_THREADS ? (int)(N - n0) : SIM_THREADS;
    for (int e = tid; e < rows * p.L; e += SIM_THREADS) {
        const int r = e / p.L, l = e - r * p.L;
        x[(n0 + r) * ldx + l] = s_acc[l * SIM_THREADS + r];
    }
}

}  // namespace

extern "C" int abc_feng_input(const double beta[3], const double kappa[3], double c[3], double a0[3], double a1[3],
                              double a2[3]) {
    vpet::clear_error();
    VPET_ARG(beta && kappa && c && a0 && a1 && a2, "abc_feng_input: null pointer");
    // (beta1 t - beta2 - beta3) e^{-k1 t} + beta2 e^{-k2 t} + beta3 e^{-k3 t}
    c[0] = kappa[0]; a0[0] = -beta[1] - beta[2]; a1[0] = beta[0]; a2[0] = 0.0;
    c[1] = kappa[1]; a0[1] = beta[1]; a1[1] = 0.0; a2[1] = 0.0;
    c[2] = kappa[2]; a0[2] = beta[2]; a1[2] = 0.0; a2[2] = 0.0;
    return ABC_OK;
}

// Validates the schedule / input and fills the kernel parameter block.
static int build_sim_params(int32_t model, const abc_frames* fr, const abc_polyexp* in, int32_t ldtheta,
                            SimParams* out) {
    VPET_ARG(fr && in && fr->t_start && fr->t_end, "abc_simulate: null frames");
    VPET_ARG(in->c && in->a0 && in->a1 && in->a2, "abc_simulate: null input arrays");
    VPET_ARG(fr->L >= 1 && fr->L <= SIM_MAXL, "abc_simulate: L must be in 1..%d", SIM_MAXL);
    VPET_ARG(in->n_terms >= 1 && in->n_terms <= SIM_MAXT, "abc_simulate: n_terms must be in 1..%d", SIM_MAXT);
    static const int need_p[4] = {4, 5, 3, 7};
    VPET_ARG(model >= 0 && model <= 3, "abc_simulate: unknown model %d", model);
    VPET_ARG(ldtheta >= need_p[model], "abc_simulate: ldtheta < parameters of model");
    SimParams& p = *out;
    memset(&p, 0, sizeof p);
    p.L = fr->L;
    double prev_end = 0.0;
    for (int l = 0; l < p.L; ++l) {
        const double ts = fr->t_start[l], te = fr->t_end[l];
        VPET_ARG(ts >= 0.0 && te > ts, "abc_simulate: frame %d has t_end <= t_start or t_start < 0", l);
        VPET_ARG(ts >= prev_end - 1e-12, "abc_simulate: frames must be ordered and non-overlapping");
        prev_end = te;
        p.ts[l] = (float)ts;
        p.dt[l] = (float)(te - ts);
    }
    p.nseg = 0;
    for (int l = 0; l < p.L; ++l)
        if (l == 0 || p.dt[l] != p.dt[l - 1]) p.seg_begin[p.nseg++] = l;
    p.seg_begin[p.nseg] = p.L;
    p.nterms = in->n_terms;
    for (int i = 0; i < in->n_terms; ++i) {
        VPET_ARG(in->c[i] >= 0.0, "abc_simulate: input rate c[%d] < 0", i);
        p.c[i] = (float)in->c[i];
        p.a[i][0] = (float)in->a0[i];
        p.a[i][1] = (float)in->a1[i];
        p.a[i][2] = (float)(2.0 * in->a2[i]);
    }
    p.lp_h = 1.0f / 16.0f;
    return ABC_OK;
}

extern "C" int abc_simulate(int32_t model, const abc_frames* fr, const abc_polyexp* in, const float* theta_dev,
                            int64_t N, int32_t ldtheta, float* x_dev, int32_t ldx, void* stream) {
    vpet::clear_error();
    SimParams p;
    const int rc = build_sim_params(model, fr, in, ldtheta, &p);
    if (rc != ABC_OK) return rc;
    VPET_ARG(N >= 0, "abc_simulate: negative N");
    VPET_ARG(N == 0 || (theta_dev && x_dev), "abc_simulate: null device pointer");
    VPET_ARG(ldx >= fr->L, "abc_simulate: ldx < L");
    if (N == 0) return ABC_OK;
    if (model == ABC_LPNTPET) {
        const double tend = (double)fr->t_end[fr->L - 1];
        const double nt = floor(tend / (double)p.lp_h) + 1.0;
        p.lp_ntab = nt < SIM_MAX_TAB ? (int)nt : SIM_MAX_TAB;
    }
    const size_t smem = ((size_t)p.L * SIM_THREADS + (size_t)p.lp_ntab) * sizeof(float);
    const unsigned grid = (unsigned)vpet_ceil_div(N, SIM_THREADS);
    cudaStream_t s = (cudaStream_t)stream;
    switch (model) {
        case ABC_2TCM_IRR: k_simulate<ABC_2TCM_IRR><<<grid, SIM_THREADS, smem, s>>>(p, theta_dev, N, ldtheta, x_dev, ldx); break;
        case ABC_2TCM_REV: k_simulate<ABC_2TCM_REV><<<grid, SIM_THREADS, smem, s>>>(p, theta_dev, N, ldtheta, x_dev, ldx); break;
        case ABC_MRTM: k_simulate<ABC_MRTM><<<grid, SIM_THREADS, smem, s>>>(p, theta_dev, N, ldtheta, x_dev, ldx); break;
        default: k_simulate<ABC_LPNTPET><<<grid, SIM_THREADS, smem, s>>>(p, theta_dev, N, ldtheta, x_dev, ldx); break;
    }
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}
