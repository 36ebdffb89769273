// Seeded random streams of libbootmmpm: keys (Algorithm 1 REQUIRE block)
// and LWE encryptions (Section 2 item (8)) drawn from a 64-bit seed.
//
// Generator: Philox4x32-10 (J. Salmon, M. Moraes, R. Dror, D. Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 128-bit counter
// is scrambled under a 64-bit key by ten rounds of two 32 x 32-bit
// multiplications and XORs, the key advancing by two Weyl constants between
// rounds.  Being counter based, any element of any stream is computed on its
// own, by a host loop or by the GPU thread that needs it.
//
// Stream layout: element i of quantity `kind` in `domain` is the block
//   philox(counter = (i mod 2^32, i >> 32, domain, kind),
//          key     = (seed mod 2^32, seed >> 32)),
// with kinds and element indices
//   1 LWE secret s_k         i = k                                   domain 0
//   2 RLWE secret z_i        i = i                                   domain N
//   3 BSK mask               i = ((k 2 + sgn) 2 l_B + row) N + c      domain N
//   4 BSK error              the same i                              domain N
//   5 KSK mask               i = r n + c, r = (i_N l_ks + j)(B_ks-1) + v-1, domain N
//   6 KSK error              i = r                                   domain N
//   7 encryption mask        i = ct n + c                            domain 0
//   8 encryption error       i = ct                                  domain 0
// and values taken from the block (w0, w1, w2, w3) as
//   uniform mod M   (w0 + w1 2^32 + w2 2^64 + w3 2^96) mod M,
//   ternary         floor(3 w0 / 2^32) - 1,   binary  floor(2 w0 / 2^32),
//   error           the discrete Gaussian exp(-k^2 / (2 sigma^2)) on
//                   [-41, 41], by inversion of its 64-bit cumulative table
//                   at r = w0 + w1 2^32 (make_cdt).
#pragma once
#include <cmath>
#include <cstdint>

namespace rng {

enum Kind : uint32_t {
    kLweSecret = 1,
    kRlweSecret = 2,
    kBskMask = 3,
    kBskErr = 4,
    kKskMask = 5,
    kKskErr = 6,
    kEncMask = 7,
    kEncErr = 8,
};

constexpr int kErrCut = 41;

struct Block {
    uint32_t w[4];
};

__host__ __device__ __forceinline__ void mulhilo(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo) {
    const uint64_t p = (uint64_t)a * b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

__host__ __device__ __forceinline__ Block philox4x32_10(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3,
                                                        uint32_t key0, uint32_t key1) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; round++) {
        if (round) {
            key0 += kWeylA;
            key1 += kWeylB;
        }
        uint32_t ha, la, hb, lb;
        mulhilo(kMulA, x0, ha, la);
        mulhilo(kMulB, x2, hb, lb);
        const uint32_t y0 = hb ^ x1 ^ key0, y2 = ha ^ x3 ^ key1;
        x0 = y0;
        x1 = lb;
        x2 = y2;
        x3 = la;
    }
    return Block{{x0, x1, x2, x3}};
}

__host__ __device__ __forceinline__ Block element(uint64_t seed, uint32_t kind, uint32_t domain, uint64_t i) {
    return philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), domain, kind, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__host__ __device__ __forceinline__ uint64_t uniform_mod(const Block &b, uint64_t M) {
    typedef unsigned __int128 u128;
    const uint64_t lo = (uint64_t)b.w[0] | ((uint64_t)b.w[1] << 32);
    const uint64_t hi = (uint64_t)b.w[2] | ((uint64_t)b.w[3] << 32);
    return (uint64_t)((((u128)hi << 64) | lo) % M);
}

__host__ __device__ __forceinline__ int ternary(const Block &b) {
    return (int)(((uint64_t)b.w[0] * 3u) >> 32) - 1;
}

__host__ __device__ __forceinline__ int binary(const Block &b) { return (int)(b.w[0] >> 31); }

// T[j] = floor(2^64 F_j) (saturated at 2^64 - 1), F_j the discrete Gaussian's
// mass on [-41, -41 + j], j in [0, 82); sums in double, from -41 upward.
struct Cdt {
    uint64_t T[2 * kErrCut];
};

inline void make_cdt(double sigma, Cdt &c) {
    double w[2 * kErrCut + 1], total = 0.0;
    const double two_var = 2.0 * sigma * sigma;
    for (int k = -kErrCut; k <= kErrCut; k++) {
        w[k + kErrCut] = std::exp(-(double)(k * k) / two_var);
        total += w[k + kErrCut];
    }
    double run = 0.0;
    for (int j = 0; j < 2 * kErrCut; j++) {
        run += w[j];
        const double scaled = std::ldexp(run / total, 64);
        c.T[j] = scaled >= 18446744073709551615.0 ? ~0ull : (uint64_t)scaled;
    }
}

__host__ __device__ __forceinline__ int gaussian(const Block &b, const Cdt &c) {
    const uint64_t r = (uint64_t)b.w[0] | ((uint64_t)b.w[1] << 32);
    int e = -kErrCut;
#pragma unroll 2
    for (int j = 0; j < 2 * kErrCut; j++) e += r >= c.T[j] ? 1 : 0;
    return e;
}

}  // namespace rng
