// Negacyclic number-theoretic transform over Z_Q on one thread block.
//
// Forward: Cooley-Tukey butterflies with the merged twist, twiddle
// psi^bitrev(k) for the k-th butterfly group (psi a primitive 2N-th root of
// unity), natural-order input, bit-reversed output:
//   NTT(a)_i = a(psi^(2 bitrev(i) + 1)).
// Inverse: Gentleman-Sande butterflies with psi^-bitrev(k), bit-reversed
// input, natural-order output, WITHOUT the final N^-1 scaling (callers fold
// N^-1 into one operand).  References: Longa and Naehrig, "Speeding up the
// number theoretic transform for faster ideal lattice-based cryptography"
// (CANS 2016); Poeppelmann, Oder and Gueneysu (LATINCRYPT 2015).
//
// `cnt` polynomials of length N = 2^logN lie back to back in shared memory.
// Values enter and leave in [0, Q).  Every stage ends with __syncthreads().
#pragma once
#include "modarith.cuh"

__device__ __forceinline__ void cta_ntt_fwd(u64 *buf, u32 cnt, u32 logN, const u64 *__restrict__ tw,
                                            const u64 *__restrict__ twsh, u64 Q) {
    const u32 half = 1u << (logN - 1);
    const u32 total = cnt << (logN - 1);
    for (u32 s = 0; s < logN; s++) {
        const u32 logLen = logN - 1 - s;
        const u32 len = 1u << logLen;
        const u32 mgrp = 1u << s;
        for (u32 b = threadIdx.x; b < total; b += blockDim.x) {
            const u32 p = b >> (logN - 1);
            const u32 bf = b & (half - 1);
            const u32 i = bf >> logLen;
            const u32 j = bf & (len - 1);
            const u32 idx = (p << logN) + (i << (logLen + 1)) + j;
            const u64 W = __ldg(tw + mgrp + i), Wsh = __ldg(twsh + mgrp + i);
            const u64 U = buf[idx];
            const u64 V = mul_shoup(buf[idx + len], W, Wsh, Q);
            buf[idx] = add_mod(U, V, Q);
            buf[idx + len] = sub_mod(U, V, Q);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void cta_ntt_inv(u64 *buf, u32 cnt, u32 logN, const u64 *__restrict__ itw,
                                            const u64 *__restrict__ itwsh, u64 Q) {
    const u32 half = 1u << (logN - 1);
    const u32 total = cnt << (logN - 1);
    for (u32 s = 0; s < logN; s++) {
        const u32 logLen = s;
        const u32 len = 1u << logLen;
        const u32 h = half >> s;
        for (u32 b = threadIdx.x; b < total; b += blockDim.x) {
            const u32 p = b >> (logN - 1);
            const u32 bf = b & (half - 1);
            const u32 i = bf >> logLen;
            const u32 j = bf & (len - 1);
            const u32 idx = (p << logN) + (i << (logLen + 1)) + j;
            const u64 W = __ldg(itw + h + i), Wsh = __ldg(itwsh + h + i);
            const u64 U = buf[idx];
            const u64 V = buf[idx + len];
            buf[idx] = add_mod(U, V, Q);
            buf[idx + len] = mul_shoup(U + Q - V, W, Wsh, Q);
        }
        __syncthreads();
    }
}
