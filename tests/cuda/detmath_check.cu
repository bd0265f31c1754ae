// Exhaustive checks of the branch-free forms of the kernels' deterministic
// math against the plain forms that the CPU oracle also follows:
//  - div_log_range(m - 1, m + 1) equals IEEE division (__fdiv_rn) for every
//    m that det_logf produces (all 2^23 mantissas, both halves of the range);
//  - det_expf (shifter rounding, selects) equals the form with rintf and an
//    early return, for every float y in [-88, 0] and a sweep outside it;
//  - div_rn_pos equals __fdiv_rn on the samplers' division ranges: every
//    normal divisor of the range with 24 dividends spread over theirs (race
//    keys E / w, multiplicity E1 / -ln(1 - p)), and S 2^-32 / k for every
//    k <= 128 with every 5th dividend;
//  - u64_to_f32_rn equals __ull2float_rn on 2^30 hashed values of every
//    magnitude and on every rounding case (just below, at and above each
//    half-way point) of every shift.
// Prints "mismatches <count>" and exits 0 when the program itself ran.
#include <cstdio>
#include <cstdint>

#include "pns_sampler.cuh"

using namespace pnsk;

__device__ float expf_plain(float y) {
    if (!(y >= -87.0f)) return 0.0f;
    const float nf = rintf(__fmul_rn(y, 0x1.715476p+0f));
    float r = __fsub_rn(y, __fmul_rn(nf, 0x1.62e400p-1f));
    r = __fsub_rn(r, __fmul_rn(nf, 0x1.7f7d1cp-20f));
    float p = 0x1.a01a02p-13f;
    p = __fadd_rn(0x1.6c16c2p-10f, __fmul_rn(r, p));
    p = __fadd_rn(0x1.111112p-7f, __fmul_rn(r, p));
    p = __fadd_rn(0x1.555556p-5f, __fmul_rn(r, p));
    p = __fadd_rn(0x1.555556p-3f, __fmul_rn(r, p));
    p = __fadd_rn(0.5f, __fmul_rn(r, p));
    p = __fadd_rn(1.0f, __fmul_rn(r, p));
    p = __fadd_rn(1.0f, __fmul_rn(r, p));
    return __fmul_rn(p, pow2f(__float2int_rn(nf)));
}

__global__ void check_div(unsigned long long *bad) {
    unsigned long long nb = 0;
    for (uint32_t mant = blockIdx.x * blockDim.x + threadIdx.x; mant < (1u << 23); mant += gridDim.x * blockDim.x) {
        const float m0 = __uint_as_float(0x3F800000u | mant);
        const float ms[2] = {m0, __fmul_rn(m0, 0.5f)};
        for (int h = 0; h < 2; ++h) {
            const float m = ms[h];
            const float x = __fsub_rn(m, 1.0f), y = __fadd_rn(m, 1.0f);
            if (__float_as_uint(div_log_range(x, y)) != __float_as_uint(__fdiv_rn(x, y))) nb++;
        }
    }
    atomicAdd(bad, nb);
}

__global__ void check_exp(unsigned long long *bad) {
    unsigned long long nb = 0;
    // every non-positive float down to -88 (bit patterns 0x80000000 .. 0xC2B00000)
    for (uint32_t u = 0x80000000u + blockIdx.x * blockDim.x + threadIdx.x; u <= 0xC2B00000u;
         u += gridDim.x * blockDim.x) {
        const float y = __uint_as_float(u);
        if (__float_as_uint(det_expf(y)) != __float_as_uint(expf_plain(y))) nb++;
    }
    // zero, positives up to 1e-3 (not used, but the forms agree there too) and below -88
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (1 << 20); i += gridDim.x * blockDim.x) {
        const float y = -88.0f - __int2float_rn(i) * 0.01f;
        if (__float_as_uint(det_expf(y)) != __float_as_uint(expf_plain(y))) nb++;
    }
    atomicAdd(bad, nb);
}

__device__ float spread(int i, int n, int elo, int ehi, uint32_t salt) {
    // dividend i of n: exponent stepped over [elo, ehi), hashed mantissa
    uint32_t h = (static_cast<uint32_t>(i) + 1u) * 2654435761u ^ salt;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    const int e = elo + (ehi - elo) * i / n;
    return __uint_as_float((static_cast<uint32_t>(e + 127) << 23) | (h & 0x007FFFFFu));
}

// every divisor with exponent in [eblo, ebhi) against NA dividends in
// [2^ealo, 2^eahi); compared where the IEEE quotient is below `cap`, and
// elsewhere the fast quotient must not fall below cap either (NaN counts as
// not below)
__global__ void check_div_pos(int eblo, int ebhi, int ealo, int eahi, float cap, unsigned long long *bad,
                              unsigned long long *count) {
    constexpr int NA = 24;
    unsigned long long nb = 0, nc = 0;
    const uint32_t total = static_cast<uint32_t>(ebhi - eblo) << 23;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int e = eblo + static_cast<int>(idx >> 23);
        const float y = __uint_as_float((static_cast<uint32_t>(e + 127) << 23) | (idx & 0x007FFFFFu));
        for (int i = 0; i < NA; ++i) {
            const float x = spread(i, NA, ealo, eahi, 0x9E3779B9u);
            const float ref = __fdiv_rn(x, y);
            const float got = div_rn_pos(x, y);
            if (ref < cap) {
                nc++;
                if (__float_as_uint(got) != __float_as_uint(ref)) nb++;
            } else if (got < cap) {
                nb++;
            }
        }
    }
    atomicAdd(bad, nb);
    atomicAdd(count, nc);
}

// S 2^-32 / k: every k in 1..128, every 5th float in [2^-32, 2^8)
__global__ void check_div_k(unsigned long long *bad, unsigned long long *count) {
    unsigned long long nb = 0, nc = 0;
    const uint32_t lo = 0x2F800000u, hi = 0x43800000u;  // 2^-32, 2^8
    for (uint32_t u = lo + 5u * (blockIdx.x * blockDim.x + threadIdx.x); u < hi; u += 5u * gridDim.x * blockDim.x) {
        const float x = __uint_as_float(u);
        for (int k = 1; k <= 128; ++k) {
            const float y = __int2float_rn(k);
            nc++;
            if (__float_as_uint(div_rn_pos(x, y)) != __float_as_uint(__fdiv_rn(x, y))) nb++;
        }
    }
    atomicAdd(bad, nb);
    atomicAdd(count, nc);
}

__device__ uint64_t mix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

__global__ void check_u64(unsigned long long *bad, unsigned long long *count) {
    unsigned long long nb = 0, nc = 0;
    for (uint64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (1ull << 30); i += gridDim.x * blockDim.x) {
        const uint64_t v = mix64(i) >> (i & 63);
        nc++;
        if (__float_as_uint(u64_to_f32_rn(v)) != __float_as_uint(__ull2float_rn(v))) nb++;
        // rounding cases: a 24-bit top shifted by s, plus the dropped part at
        // half - 1, half, half + 1 (and 0)
        const int sh = 1 + static_cast<int>(i % 40);
        const uint64_t top = (mix64(i + 0x9e37ull) & 0x7FFFFFull) | 0x800000ull;
        const uint64_t half = 1ull << (sh - 1);
        const uint64_t base = top << sh;
        const uint64_t cases[4] = {base, base + half - 1, base + half, base + half + 1};
        for (int c = 0; c < 4; ++c) {
            nc++;
            if (__float_as_uint(u64_to_f32_rn(cases[c])) != __float_as_uint(__ull2float_rn(cases[c]))) nb++;
        }
    }
    atomicAdd(bad, nb);
    atomicAdd(count, nc);
}

int main() {
    unsigned long long *d, h[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (cudaMalloc(&d, 80) != cudaSuccess) return 2;
    cudaMemset(d, 0, 80);
    check_div<<<608, 256>>>(d);
    check_exp<<<1216, 256>>>(d + 1);
    // race keys: E in [2^-56, 2^5), every normal w in [2^-126, 2); keys at or
    // above 3e38 (never the least: the anchor's key is E <= 16.7) need only stay there
    check_div_pos<<<1216, 256>>>(-126, 1, -56, 5, 3.0e38f, d + 2, d + 3);
    // multiplicity: E1 in [2^-25, 2^6), every normal -ln(1 - p) in [2^-126, 2^6);
    // exact below 2^63 (the saturation bound), at or above it elsewhere
    check_div_pos<<<1216, 256>>>(-126, 6, -25, 6, 0x1p63f, d + 4, d + 5);
    check_div_k<<<1216, 256>>>(d + 6, d + 7);
    check_u64<<<1216, 256>>>(d + 8, d + 9);
    if (cudaDeviceSynchronize() != cudaSuccess) return 3;
    cudaMemcpy(h, d, 80, cudaMemcpyDeviceToHost);
    printf("div_mismatches %llu\nexp_mismatches %llu\n", h[0], h[1]);
    printf("race_div_mismatches %llu\nrace_div_compared %llu\n", h[2], h[3]);
    printf("mult_div_mismatches %llu\nmult_div_compared %llu\n", h[4], h[5]);
    printf("k_div_mismatches %llu\nk_div_compared %llu\n", h[6], h[7]);
    printf("u64_mismatches %llu\nu64_compared %llu\n", h[8], h[9]);
    return 0;
}
