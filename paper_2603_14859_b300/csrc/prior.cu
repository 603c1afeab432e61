// Prior draws (Algorithm 1, steps 1-2): uniform boxes from a counter-based
// Philox4x32-10 stream (Salmon et al., SC'11), so every draw is a pure function
// of (seed, model, global draw index, parameter) and can be regenerated anywhere.
#include "common.cuh"

namespace {

struct Box {
    double lo[8];
    double span[8];
};

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0,
                                             uint32_t k1) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
}

// Ten rounds, key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        philox_round(c.x, c.y, c.z, c.w, k0, k1);
    }
    return c;
}

// One thread per draw; a draw needs ceil(P/4) Philox blocks.
__global__ void k_sample_prior(uint64_t seed, int model, Box box, int P, int64_t N, int64_t first, float* theta,
                               int ld) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const uint64_t g = (uint64_t)(first + n);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    float out[8];
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        if (blk * 4 >= P) break;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), (uint32_t)model, (uint32_t)blk),
                                      k0, k1);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int p = blk * 4 + q;
            if (p < P) {
                const double u = (double)(w[q] >> 8) * (1.0 / 16777216.0);
                // lo + span * u in fp64 with explicit rounding steps (no fused multiply-add),
                // then one rounding to fp32.
                out[p] = (float)__dadd_rn(box.lo[p], __dmul_rn(box.span[p], u));
            }
        }
    }
    float* row = theta + n * ld;
    for (int p = 0; p < P; ++p) row[p] = out[p];
}

}  // namespace

extern "C" int abc_sample_prior(uint64_t seed, int32_t model, const double* lo, const double* hi, int32_t P,
                                int64_t N, int64_t first_index, float* theta_dev, int32_t ldtheta, void* stream) {
    vpet::clear_error();
    VPET_ARG(lo && hi && theta_dev, "abc_sample_prior: null pointer");
    VPET_ARG(P >= 1 && P <= 8, "abc_sample_prior: P must be in 1..8 (got %d)", P);
    VPET_ARG(ldtheta >= P, "abc_sample_prior: ldtheta < P");
    VPET_ARG(N >= 0 && first_index >= 0, "abc_sample_prior: negative N or first_index");
    VPET_ARG(model >= 0, "abc_sample_prior: negative model id");
    Box b;
    for (int p = 0; p < 8; ++p) {
        b.lo[p] = p < P ? lo[p] : 0.0;
        // span computed exactly as the definition: hi - lo in fp64
        b.span[p] = p < P ? hi[p] - lo[p] : 0.0;
        if (p < P) VPET_ARG(hi[p] >= lo[p], "abc_sample_prior: hi < lo for parameter %d", p);
    }
    if (N == 0) return ABC_OK;
    const int threads = 256;
    k_sample_prior<<<(unsigned)vpet_ceil_div(N, threads), threads, 0, (cudaStream_t)stream>>>(
        seed, model, b, P, N, first_index, theta_dev, ldtheta);
    VPET_LAUNCH_CHECK();
    return ABC_OK;
}
