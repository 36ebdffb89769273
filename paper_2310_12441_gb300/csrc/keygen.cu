// Key generation on the GPU, client-side LWE encryption and decryption,
// and the small host utilities of libbootmmpm.
//
// Bootstrapping keys (Algorithm 1 REQUIRE; Section 2 item (14)): for every
// LWE coordinate k and both signs, an RGSW encryption under z of
// s_k+ = max(s_k, 0) or s_k- = max(-s_k, 0).  Rows are built straight in the
// NTT domain: with a^ = NTT(a), z^ = NTT(z), e^ = NTT(e) and the constant
// mu B^j (whose transform is mu B^j in every slot),
//   row j       : ( a^ + mu B^j ,  a^ z^ + e^          ) * N^-1
//   row l_B + j : ( a^          ,  a^ z^ + e^ + mu B^j ) * N^-1.
// Key-switching keys (Section 2 item (11)): LWE_{n,Q} encryptions under s of
// v z_i g_j for the approximate gadget g_j = floor((Q B_ks^j + P/2) / P).
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "ntt.cuh"
#include "philox.cuh"

typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// Host arithmetic (setup only)
// ---------------------------------------------------------------------------

u64 host_mulmod(u64 a, u64 b, u64 Q) { return (u64)((u128)a * b % Q); }

static u64 host_powmod(u64 a, u64 e, u64 Q) {
    u64 r = 1 % Q;
    a %= Q;
    while (e) {
        if (e & 1) r = host_mulmod(r, a, Q);
        a = host_mulmod(a, a, Q);
        e >>= 1;
    }
    return r;
}

// Deterministic Miller-Rabin for 64-bit integers (the first 12 primes as
// bases suffice below 3.3e24).
static bool host_is_prime(u64 n) {
    if (n < 2) return false;
    static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : bases) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (u64 a : bases) {
        u64 x = host_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r; i++) {
            x = host_mulmod(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

static u64 shoup_of(u64 w, u64 Q) { return (u64)(((u128)w << 64) / Q); }

static u32 bitrev(u32 x, u32 bits) {
    u32 r = 0;
    for (u32 i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

bm_status bm_check_key_params(const bm_key_params *p) {
    if (!p) return BM_EINVAL;
    if (p->N < 256 || p->N > BM_MAX_N || (p->N & (p->N - 1))) return BM_EINVAL;
    if (p->n == 0 || p->n > 4096) return BM_EINVAL;
    if (p->l_B < 2 || p->l_B > BM_MAX_L_B || p->log2_B == 0 || p->log2_B > 32) return BM_EINVAL;
    if (p->log2_Bks == 0 || p->log2_Bks > 8 || p->l_ks == 0 || p->l_ks > 16 ||
        p->log2_Bks * p->l_ks > 40)
        return BM_EINVAL;
    if (p->Q < 3 || p->Q >= (1ull << 61)) return BM_EINVAL;
    if ((u64)p->log2_B * p->l_B < 64 && (1ull << (p->log2_B * p->l_B)) < p->Q) return BM_EINVAL;
    if ((1ull << (p->log2_Bks * p->l_ks)) >= p->Q) return BM_EINVAL;
    // 2 signs x 2 l_B products below Q^2 must not overflow the 128-bit MAC.
    u128 q2 = (u128)(p->Q - 1) * (p->Q - 1);
    if (q2 > (~(u128)0) / (4u * p->l_B)) return BM_EINVAL;
    if (!host_is_prime(p->Q) || (p->Q - 1) % (2ull * p->N)) return BM_ENOTPRIME;
    return BM_OK;
}

// ---------------------------------------------------------------------------
// Device kernels
// ---------------------------------------------------------------------------

// Forward NTT of `count` polynomials (given as signed int8 or uint64 words).
__global__ void k_ntt_z(const int8_t *__restrict__ z, u64 *__restrict__ zhat, KeyDev K) {
    extern __shared__ u64 sm[];
    const u64 Q = K.mq.Q;
    for (u32 i = threadIdx.x; i < K.N; i += blockDim.x) {
        int v = z[i];
        sm[i] = v >= 0 ? (u64)v : Q - (u64)(-v);
    }
    __syncthreads();
    cta_ntt_fwd(sm, 1, K.logN, K.tw, K.twsh, Q);
    for (u32 i = threadIdx.x; i < K.N; i += blockDim.x) zhat[i] = sm[i];
}

// RGSW row `row_id` (absolute index into [n][2][2 l_B]) from its mask
// (sm[0, N)) and error (sm[N, 2N), in Z_Q), both in the coefficient domain;
// the whole block calls it (see the file header for the formula).
__device__ void bsk_row_finish(u64 *sm, size_t row_id, const int8_t *__restrict__ s,
                               const u64 *__restrict__ zhat, u64 *__restrict__ bsk, const KeyDev &K) {
    const u32 N = K.N, lB = K.l_B;
    const u64 Q = K.mq.Q;
    __syncthreads();
    cta_ntt_fwd(sm, 2, K.logN, K.tw, K.twsh, Q);
    const u32 row = (u32)(row_id % (2 * lB));
    const u32 sgn = (u32)((row_id / (2 * lB)) % 2);
    const size_t k = row_id / (4 * lB);
    const int sk = s[k];
    const bool mu = sgn == 0 ? sk > 0 : sk < 0;
    u64 g = 0;
    if (mu) {
        // B^j mod Q, j = row mod l_B (B^j may exceed Q only for j*log2_B >= 61)
        u64 gg = 1 % Q;
        for (u32 d = 0; d < row % lB; d++) {
            u64 lo = 0, hi = 0;
            mac128(lo, hi, gg, 1ull << K.log2_B);
            gg = reduce128(lo, hi, K.mq);
        }
        g = gg;
    }
    const u64 g0 = row < lB ? g : 0, g1 = row < lB ? 0 : g;
    u64 *o = bsk + row_id * 2 * N;
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
        const u64 ah = sm[i], eh = sm[N + i];
        u64 lo = 0, hi = 0;
        mac128(lo, hi, ah, zhat[i]);
        add128(lo, hi, eh);
        add128(lo, hi, g1);
        const u64 c1 = reduce128(lo, hi, K.mq);
        const u64 c0 = add_mod(ah, g0, Q);
        // stored split into the multiply-accumulate's limbs (KeyDev::lbits):
        // per position the low limbs of both columns, then their high limbs
        const u64 lmask = (1ull << K.lbits) - 1;
        const u64 w0 = mul_shoup(c0, K.ninv, K.ninv_sh, Q), w1 = mul_shoup(c1, K.ninv, K.ninv_sh, Q);
        o[2 * i] = (w0 & lmask) | ((w1 & lmask) << 32);
        o[2 * i + 1] = (w0 >> K.lbits) | ((w1 >> K.lbits) << 32);
    }
}

__device__ __forceinline__ u64 signed_to_zq(int v, u64 Q) { return v >= 0 ? (u64)v : Q - (u64)(-v); }

// One RGSW row per block from caller-supplied randomness: mask/err hold the
// rows [row0, row0 + gridDim.x).
__global__ void k_bsk_rows(const u64 *__restrict__ mask, const int8_t *__restrict__ err,
                           const int8_t *__restrict__ s, const u64 *__restrict__ zhat,
                           u64 *__restrict__ bsk, KeyDev K, size_t row0) {
    extern __shared__ u64 sm[];
    const u32 N = K.N;
    const u64 *a = mask + (size_t)blockIdx.x * N;
    const int8_t *e = err + (size_t)blockIdx.x * N;
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
        sm[i] = a[i];
        sm[N + i] = signed_to_zq(e[i], K.mq.Q);
    }
    bsk_row_finish(sm, row0 + blockIdx.x, s, zhat, bsk, K);
}

// One RGSW row per block, its mask and error drawn from the seed's streams
// (kinds 3 and 4, element index row N + i, domain N).
__global__ void k_bsk_rows_seeded(uint64_t seed, rng::Cdt cdt, const int8_t *__restrict__ s,
                                  const u64 *__restrict__ zhat, u64 *__restrict__ bsk, KeyDev K,
                                  size_t row0) {
    extern __shared__ u64 sm[];
    const u32 N = K.N;
    const size_t row_id = row0 + blockIdx.x;
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
        const uint64_t idx = (uint64_t)row_id * N + i;
        sm[i] = rng::uniform_mod(rng::element(seed, rng::kBskMask, N, idx), K.mq.Q);
        sm[N + i] = signed_to_zq(rng::gaussian(rng::element(seed, rng::kBskErr, N, idx), cdt), K.mq.Q);
    }
    bsk_row_finish(sm, row_id, s, zhat, bsk, K);
}

// Ring degrees above BM_MAX_N_BLOCK (one block cannot transform a row): the
// rows' masks and errors in Z_Q, [rows][N], for the two-pass transforms of
// big.cu; seeded (the same streams and indices as k_bsk_rows_seeded) or from
// caller randomness (errors as int8).
__global__ void k_big_rows_seeded(uint64_t seed, rng::Cdt cdt, u64 *__restrict__ a, u64 *__restrict__ e, u32 N,
                                  u64 Q, size_t row0) {
    const size_t r = blockIdx.y;
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const uint64_t idx = (uint64_t)(row0 + r) * N + i;
        a[r * N + i] = rng::uniform_mod(rng::element(seed, rng::kBskMask, N, idx), Q);
        e[r * N + i] = signed_to_zq(rng::gaussian(rng::element(seed, rng::kBskErr, N, idx), cdt), Q);
    }
}
__global__ void k_big_rows_given(const int8_t *__restrict__ err, u64 *__restrict__ e, size_t words, u64 Q) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x)
        e[i] = signed_to_zq(err[i], Q);
}
__global__ void k_big_z(const int8_t *__restrict__ z, u64 *__restrict__ zq, u32 N, u64 Q) {
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        zq[i] = signed_to_zq(z[i], Q);
}

struct KsGadget { u64 g[16]; };

// Key-switching row `row` = (i, j, v) by one warp: (a', <a', s> + e + v z_i g_j)
// with mask word c given by get_a(c).
template <typename GetA>
__device__ __forceinline__ void ksk_row(size_t row, GetA get_a, int ev, const int8_t *__restrict__ s,
                                        const int8_t *__restrict__ z, u64 *__restrict__ ksk, const KeyDev &K,
                                        const KsGadget &G) {
    const u32 lane = threadIdx.x & 31;
    const u32 n = K.n, B1 = (1u << K.log2_Bks) - 1;
    const u64 Q = K.mq.Q;
    u64 *o = ksk + row * (n + 1);
    u64 lo = 0, hi = 0;
    for (u32 c = lane; c < n; c += 32) {
        const u64 x = get_a(c);
        o[c] = x;
        const int sc = s[c];
        if (sc > 0) add128(lo, hi, x);
        else if (sc < 0) add128(lo, hi, Q - x);
    }
    u64 acc = reduce128(lo, hi, K.mq);
    for (int off = 16; off; off >>= 1) acc = add_mod(acc, __shfl_down_sync(0xffffffffu, acc, off), Q);
    if (lane == 0) {
        const u32 v = (u32)(row % B1) + 1;
        const u32 j = (u32)((row / B1) % K.l_ks);
        const u32 i = (u32)(row / ((size_t)B1 * K.l_ks));
        u64 l2 = 0, h2 = 0;
        mac128(l2, h2, v, G.g[j]);
        u64 vg = reduce128(l2, h2, K.mq);
        const int zi = z[i];
        u64 msg = zi > 0 ? vg : (zi < 0 ? (vg ? Q - vg : 0) : 0);
        o[n] = add_mod(add_mod(acc, signed_to_zq(ev, Q), Q), msg, Q);
    }
}

// One key-switching row per warp from caller-supplied randomness: mask holds
// rows [row0, row_end) only; err is indexed absolutely.
__global__ void k_ksk_rows(const u64 *__restrict__ mask, const int8_t *__restrict__ err,
                           const int8_t *__restrict__ s, const int8_t *__restrict__ z,
                           u64 *__restrict__ ksk, KeyDev K, KsGadget G, size_t row0,
                           size_t row_end) {
    const size_t row = row0 + (size_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (row >= row_end) return;
    const u64 *a = mask + (row - row0) * K.n;
    ksk_row(row, [&](u32 c) { return a[c]; }, err[row], s, z, ksk, K, G);
}

// One key-switching row per warp, mask and error drawn from the seed's
// streams (kinds 5 and 6, domain N).
__global__ void k_ksk_rows_seeded(uint64_t seed, rng::Cdt cdt, const int8_t *__restrict__ s,
                                  const int8_t *__restrict__ z, u64 *__restrict__ ksk, KeyDev K, KsGadget G,
                                  size_t rows) {
    const size_t row = (size_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (row >= rows) return;
    const u32 N = K.N, n = K.n;
    const u64 Q = K.mq.Q;
    const int ev = rng::gaussian(rng::element(seed, rng::kKskErr, N, row), cdt);
    ksk_row(row, [&](u32 c) { return rng::uniform_mod(rng::element(seed, rng::kKskMask, N, (uint64_t)row * n + c), Q); },
            ev, s, z, ksk, K, G);
}

// ---------------------------------------------------------------------------
// Host entry points
// ---------------------------------------------------------------------------

static void fill_keydev_constants(KeyDev &K, const bm_key_params &p, u32 logN, u64 psi) {
    const u64 Q = p.Q;
    K.mq.Q = Q;
    K.mq.two_Q = 2 * Q;
    K.mq.r64 = (u64)(((u128)1 << 64) % Q);
    K.mq.r64_sh = shoup_of(K.mq.r64, Q);
    K.mq.one_sh = shoup_of(1, Q);
    K.ninv = host_powmod(p.N, Q - 2, Q);
    K.ninv_sh = shoup_of(K.ninv, Q);
    const u64 P = 1ull << (p.log2_Bks * p.l_ks);
    K.ks_pq = shoup_of(P, Q);
    K.n = p.n;
    K.N = p.N;
    K.logN = logN;
    K.log2_B = p.log2_B;
    K.l_B = p.l_B;
    K.log2_Bks = p.log2_Bks;
    K.l_ks = p.l_ks;
    u32 fold_each = 0;
    limb_plan(p, choose_variant(p), K.lbits, fold_each);
    (void)psi;
}

static u64 find_psi(u64 Q, u32 N) {
    for (u64 g = 2; g < 1000000; g++) {
        u64 psi = host_powmod(g, (Q - 1) / (2ull * N), Q);
        if (host_powmod(psi, N, Q) == Q - 1) return psi;
    }
    return 0;
}

extern "C" void bm_free_eval_key(bm_eval_key *ek) {
    if (!ek) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ek->device);
    cudaFree(ek->d_bsk);
    cudaFree(ek->d_ksk);
    cudaFree(ek->d_tables);
    cudaFree(ek->d_view);
    cudaSetDevice(prev);
    delete ek;
}

extern "C" void bm_free_secret_key(bm_secret_key *sk) {
    if (!sk) return;
    free(sk->s);
    free(sk->z);
    delete sk;
}

extern "C" size_t bm_eval_key_bytes(const bm_eval_key *ek) { return ek ? ek->bytes : 0; }

namespace {
struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};
}  // namespace

// Where the randomness of key generation comes from: caller arrays (rnd), or
// the seed's Philox streams (rnd == nullptr).
struct KeySource {
    const bm_key_randomness *rnd;
    uint64_t seed;
    rng::Cdt cdt;
};

static bm_status keygen_impl(const bm_key_params *params, const int8_t *s, const int8_t *z,
                             const KeySource &src, bm_eval_key *ek) {
    const bm_key_params &p = *params;
    const u32 N = p.N, n = p.n, lB = p.l_B;
    u32 logN = 0;
    while ((1u << logN) < N) logN++;
    const u64 Q = p.Q;
    const u64 psi = find_psi(Q, N);
    if (!psi) return BM_ENOTPRIME;

    // Twiddle tables: fwd, fwd_sh, inv, inv_sh (each N words), then the same
    // as interleaved (w, w') pairs, forward and inverse (2N words each).
    std::vector<u64> tab(8 * (size_t)N);
    const u64 psi_inv = host_powmod(psi, Q - 2, Q);
    for (u32 k = 0; k < N; k++) {
        const u32 br = bitrev(k, logN);
        const u64 w = host_powmod(psi, br, Q), wi = host_powmod(psi_inv, br, Q);
        tab[k] = w;
        tab[N + k] = shoup_of(w, Q);
        tab[2 * N + k] = wi;
        tab[3 * N + k] = shoup_of(wi, Q);
        tab[4 * N + 2 * k] = w;
        tab[4 * N + 2 * k + 1] = tab[N + k];
        tab[6 * N + 2 * k] = wi;
        tab[6 * N + 2 * k + 1] = tab[3 * N + k];
    }
    const size_t bsk_words = (size_t)n * 2 * 2 * lB * 2 * N;
    const u32 B1 = (1u << p.log2_Bks) - 1;
    const size_t ksk_rows = (size_t)N * p.l_ks * B1;
    const size_t ksk_words = ksk_rows * (n + 1);

    if (cudaMalloc(&ek->d_tables, tab.size() * 8 + 8 * (size_t)N) != cudaSuccess) return BM_ENOMEM;
    if (cudaMalloc(&ek->d_bsk, bsk_words * 8) != cudaSuccess) return BM_ENOMEM;
    if (cudaMalloc(&ek->d_ksk, ksk_words * 8) != cudaSuccess) return BM_ENOMEM;
    if (cudaMalloc(&ek->d_view, sizeof(KeyDev)) != cudaSuccess) return BM_ENOMEM;
    ek->bytes = bsk_words * 8 + ksk_words * 8 + tab.size() * 8 + 8 * (size_t)N + sizeof(KeyDev);
    BM_CUDA_TRY(cudaMemcpy(ek->d_tables, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice));

    KeyDev &K = ek->host_view;
    fill_keydev_constants(K, p, logN, psi);
    K.bsk = ek->d_bsk;
    K.ksk = ek->d_ksk;
    K.tw = ek->d_tables;
    K.twsh = ek->d_tables + N;
    K.itw = ek->d_tables + 2 * N;
    K.itwsh = ek->d_tables + 3 * N;
    K.twp = ek->d_tables + 4 * N;
    K.itwp = ek->d_tables + 6 * N;
    BM_CUDA_TRY(cudaMemcpy(ek->d_view, &K, sizeof(KeyDev), cudaMemcpyHostToDevice));
    u64 *d_zhat = ek->d_tables + 8 * (size_t)N;

    // Secrets on the device.
    DevBuf d_s, d_z;
    BM_CUDA_TRY(cudaMalloc(&d_s.p, n));
    BM_CUDA_TRY(cudaMalloc(&d_z.p, N));
    BM_CUDA_TRY(cudaMemcpy(d_s.p, s, n, cudaMemcpyHostToDevice));
    BM_CUDA_TRY(cudaMemcpy(d_z.p, z, N, cudaMemcpyHostToDevice));

    const u32 threads = N / 2 < 512 ? N / 2 : 512;
    const size_t rows_per_k = 2 * 2 * (size_t)lB;
    const u32 kchunk = 64;
    if (N > BM_MAX_N_BLOCK) {
        // z^ and the RGSW rows through the two-pass transforms (big.cu)
        const unsigned zb = (N + 255) / 256;
        k_big_z<<<zb, 256>>>((const int8_t *)d_z.p, d_zhat, N, p.Q);
        BM_CUDA_TRY(cudaGetLastError());
        bm_status st = bm_big_ntt(d_zhat, 1, ek->d_view, N, false, 0);
        if (st != BM_OK) return st;
        DevBuf d_a, d_e, d_err8;
        BM_CUDA_TRY(cudaMalloc(&d_a.p, kchunk * rows_per_k * N * 8));
        BM_CUDA_TRY(cudaMalloc(&d_e.p, kchunk * rows_per_k * N * 8));
        if (src.rnd) BM_CUDA_TRY(cudaMalloc(&d_err8.p, kchunk * rows_per_k * N));
        for (u32 k0 = 0; k0 < n; k0 += kchunk) {
            const u32 k1 = k0 + kchunk < n ? k0 + kchunk : n;
            const size_t rows = (size_t)(k1 - k0) * rows_per_k, row0 = (size_t)k0 * rows_per_k;
            if (src.rnd) {
                BM_CUDA_TRY(cudaMemcpy(d_a.p, src.rnd->bsk_mask + row0 * N, rows * N * 8, cudaMemcpyHostToDevice));
                BM_CUDA_TRY(cudaMemcpy(d_err8.p, src.rnd->bsk_err + row0 * N, rows * N, cudaMemcpyHostToDevice));
                k_big_rows_given<<<4096, 256>>>((const int8_t *)d_err8.p, (u64 *)d_e.p, rows * N, p.Q);
            } else {
                k_big_rows_seeded<<<dim3(zb < 64 ? zb : 64, (unsigned)rows), 256>>>(src.seed, src.cdt, (u64 *)d_a.p,
                                                                                     (u64 *)d_e.p, N, p.Q, row0);
            }
            BM_CUDA_TRY(cudaGetLastError());
            if ((st = bm_big_ntt((u64 *)d_a.p, (u32)rows, ek->d_view, N, false, 0)) != BM_OK) return st;
            if ((st = bm_big_ntt((u64 *)d_e.p, (u32)rows, ek->d_view, N, false, 0)) != BM_OK) return st;
            if ((st = bm_big_bsk_finish((const u64 *)d_a.p, (const u64 *)d_e.p, (const int8_t *)d_s.p, d_zhat,
                                        ek->d_bsk, ek->d_view, N, row0, (u32)rows, 0)) != BM_OK)
                return st;
            BM_CUDA_TRY(cudaDeviceSynchronize());
        }
    } else {
    BM_CUDA_TRY(cudaFuncSetAttribute(k_ntt_z, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(N * 8)));
    k_ntt_z<<<1, threads, N * 8>>>((const int8_t *)d_z.p, d_zhat, K);
    BM_CUDA_TRY(cudaGetLastError());

    // Bootstrapping keys: one RGSW row per block, in chunks of key indices
    // (which bounds the staging memory of caller-supplied randomness).
    if (src.rnd) {
        DevBuf d_mask, d_err;
        BM_CUDA_TRY(cudaMalloc(&d_mask.p, kchunk * rows_per_k * N * 8));
        BM_CUDA_TRY(cudaMalloc(&d_err.p, kchunk * rows_per_k * N));
        BM_CUDA_TRY(cudaFuncSetAttribute(k_bsk_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         2 * N * 8));
        for (u32 k0 = 0; k0 < n; k0 += kchunk) {
            const u32 k1 = k0 + kchunk < n ? k0 + kchunk : n;
            const size_t rows = (size_t)(k1 - k0) * rows_per_k;
            BM_CUDA_TRY(cudaMemcpy(d_mask.p, src.rnd->bsk_mask + (size_t)k0 * rows_per_k * N,
                                   rows * N * 8, cudaMemcpyHostToDevice));
            BM_CUDA_TRY(cudaMemcpy(d_err.p, src.rnd->bsk_err + (size_t)k0 * rows_per_k * N, rows * N,
                                   cudaMemcpyHostToDevice));
            k_bsk_rows<<<(unsigned)rows, threads, 2 * N * 8>>>((const u64 *)d_mask.p, (const int8_t *)d_err.p,
                                                                (const int8_t *)d_s.p, d_zhat, ek->d_bsk, K,
                                                                (size_t)k0 * rows_per_k);
            BM_CUDA_TRY(cudaGetLastError());
            BM_CUDA_TRY(cudaDeviceSynchronize());
        }
    } else {
        BM_CUDA_TRY(cudaFuncSetAttribute(k_bsk_rows_seeded, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         2 * N * 8));
        for (u32 k0 = 0; k0 < n; k0 += kchunk) {
            const u32 k1 = k0 + kchunk < n ? k0 + kchunk : n;
            const size_t rows = (size_t)(k1 - k0) * rows_per_k;
            k_bsk_rows_seeded<<<(unsigned)rows, threads, 2 * N * 8>>>(src.seed, src.cdt, (const int8_t *)d_s.p,
                                                                       d_zhat, ek->d_bsk, K,
                                                                       (size_t)k0 * rows_per_k);
            BM_CUDA_TRY(cudaGetLastError());
        }
        BM_CUDA_TRY(cudaDeviceSynchronize());
    }
    }
    // Key-switching keys: one LWE row per warp.
    KsGadget G;
    memset(&G, 0, sizeof(G));
    const u128 P = (u128)1 << (p.log2_Bks * p.l_ks);
    for (u32 j = 0; j < p.l_ks && j < 16; j++)
        G.g[j] = (u64)((((u128)Q << (p.log2_Bks * j)) + P / 2) / P);
    if (src.rnd) {
        const size_t chunk_rows = 1u << 16;
        DevBuf d_mask, d_err;
        BM_CUDA_TRY(cudaMalloc(&d_mask.p, chunk_rows * n * 8));
        BM_CUDA_TRY(cudaMalloc(&d_err.p, ksk_rows));
        BM_CUDA_TRY(cudaMemcpy(d_err.p, src.rnd->ksk_err, ksk_rows, cudaMemcpyHostToDevice));
        for (size_t r0 = 0; r0 < ksk_rows; r0 += chunk_rows) {
            const size_t r1 = r0 + chunk_rows < ksk_rows ? r0 + chunk_rows : ksk_rows;
            BM_CUDA_TRY(cudaMemcpy(d_mask.p, src.rnd->ksk_mask + r0 * n, (r1 - r0) * n * 8,
                                   cudaMemcpyHostToDevice));
            const size_t rows = r1 - r0;
            const unsigned blocks = (unsigned)((rows + 7) / 8);
            k_ksk_rows<<<blocks, 256>>>((const u64 *)d_mask.p, (const int8_t *)d_err.p,
                                        (const int8_t *)d_s.p, (const int8_t *)d_z.p,
                                        ek->d_ksk, K, G, r0, r1);
            BM_CUDA_TRY(cudaGetLastError());
            BM_CUDA_TRY(cudaDeviceSynchronize());
        }
    } else {
        const unsigned blocks = (unsigned)((ksk_rows + 7) / 8);
        k_ksk_rows_seeded<<<blocks, 256>>>(src.seed, src.cdt, (const int8_t *)d_s.p, (const int8_t *)d_z.p,
                                           ek->d_ksk, K, G, ksk_rows);
        BM_CUDA_TRY(cudaGetLastError());
        BM_CUDA_TRY(cudaDeviceSynchronize());
    }
    return BM_OK;
}

static bm_secret_key *new_secret_key(const bm_key_params &p) {
    bm_secret_key *sk = new (std::nothrow) bm_secret_key();
    if (!sk) return nullptr;
    sk->p = p;
    sk->s = (int8_t *)malloc(p.n);
    sk->z = (int8_t *)malloc(p.N);
    if (!sk->s || !sk->z) {
        bm_free_secret_key(sk);
        return nullptr;
    }
    return sk;
}

// Builds the evaluation key on `device` for secret key sk.
static bm_status make_eval_key(const bm_key_params *params, const bm_secret_key *sk, const KeySource &src,
                               int device, bm_eval_key **ek_out) {
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return BM_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return BM_EINVAL;
    bm_eval_key *ek = new (std::nothrow) bm_eval_key();
    if (!ek) {
        cudaSetDevice(prev);
        return BM_ENOMEM;
    }
    ek->device = device;
    ek->p = *params;
    bm_status st = keygen_impl(params, sk->s, sk->z, src, ek);
    cudaSetDevice(prev);
    if (st != BM_OK) {
        bm_free_eval_key(ek);
        return st;
    }
    *ek_out = ek;
    return BM_OK;
}

extern "C" bm_status bm_keygen(const bm_key_params *params, const bm_key_randomness *rnd,
                               int device, bm_secret_key **sk_out, bm_eval_key **ek_out) {
    if (!params || !rnd || !sk_out || !ek_out || !rnd->s || !rnd->z || !rnd->bsk_mask ||
        !rnd->bsk_err || !rnd->ksk_mask || !rnd->ksk_err)
        return BM_EINVAL;
    bm_status st = bm_check_key_params(params);
    if (st != BM_OK) return st;
    for (u32 i = 0; i < params->n; i++)
        if (rnd->s[i] < -1 || rnd->s[i] > 1) return BM_EINVAL;
    for (u32 i = 0; i < params->N; i++)
        if (rnd->z[i] < -1 || rnd->z[i] > 1) return BM_EINVAL;
    bm_secret_key *sk = new_secret_key(*params);
    if (!sk) return BM_ENOMEM;
    memcpy(sk->s, rnd->s, params->n);
    memcpy(sk->z, rnd->z, params->N);
    KeySource src{rnd, 0, {}};
    st = make_eval_key(params, sk, src, device, ek_out);
    if (st != BM_OK) {
        bm_free_secret_key(sk);
        return st;
    }
    *sk_out = sk;
    return BM_OK;
}

extern "C" bm_status bm_secret_key_seeded(const bm_key_params *params, uint32_t lwe_secret, uint64_t seed,
                                          bm_secret_key **sk_out) {
    if (!params || !sk_out || lwe_secret > BM_SECRET_TERNARY) return BM_EINVAL;
    bm_status st = bm_check_key_params(params);
    if (st != BM_OK) return st;
    bm_secret_key *sk = new_secret_key(*params);
    if (!sk) return BM_ENOMEM;
    for (u32 k = 0; k < params->n; k++) {
        const rng::Block b = rng::element(seed, rng::kLweSecret, 0, k);
        sk->s[k] = (int8_t)(lwe_secret == BM_SECRET_TERNARY ? rng::ternary(b) : rng::binary(b));
    }
    for (u32 i = 0; i < params->N; i++)
        sk->z[i] = (int8_t)rng::ternary(rng::element(seed, rng::kRlweSecret, params->N, i));
    *sk_out = sk;
    return BM_OK;
}

extern "C" bm_status bm_keygen_seeded(const bm_key_params *params, uint32_t lwe_secret, double sigma,
                                      uint64_t seed, int device, bm_secret_key **sk_out,
                                      bm_eval_key **ek_out) {
    if (!params || !sk_out || !ek_out || !(sigma > 0.0) || sigma > BM_SIGMA_MAX) return BM_EINVAL;
    bm_secret_key *sk = nullptr;
    bm_status st = bm_secret_key_seeded(params, lwe_secret, seed, &sk);
    if (st != BM_OK) return st;
    KeySource src{nullptr, seed, {}};
    rng::make_cdt(sigma, src.cdt);
    st = make_eval_key(params, sk, src, device, ek_out);
    if (st != BM_OK) {
        bm_free_secret_key(sk);
        return st;
    }
    *sk_out = sk;
    return BM_OK;
}

extern "C" bm_status bm_secret_key_get(const bm_secret_key *sk, int8_t *s_out, int8_t *z_out) {
    if (!sk) return BM_EINVAL;
    if (s_out) memcpy(s_out, sk->s, sk->p.n);
    if (z_out) memcpy(z_out, sk->z, sk->p.N);
    return BM_OK;
}

// ---------------------------------------------------------------------------
// Client-side LWE encryption / decryption (Section 2 item (8))
// ---------------------------------------------------------------------------

// ct = (a, <a, s> + msg floor(q/t) + e) mod q, mask word c = mask(c) in [0, q).
template <typename Mask>
static void encrypt_one(const bm_secret_key *sk, u64 q, u32 t, u32 msg, Mask mask, int e, u64 *o) {
    const u32 n = sk->p.n;
    const u64 delta = q / t;
    u128 pos = 0, neg = 0;
    for (u32 c = 0; c < n; c++) {
        const u64 a = mask(c);
        o[c] = a;
        if (sk->s[c] > 0) pos += a;
        else if (sk->s[c] < 0) neg += a;
    }
    pos += (u128)(msg % t) * delta + (e >= 0 ? (u64)e : 0);
    neg += e < 0 ? (u64)(-e) : 0;
    const u64 pm = (u64)(pos % q), nm = (u64)(neg % q);
    o[n] = pm >= nm ? pm - nm : pm + q - nm;
}

extern "C" bm_status bm_encrypt(const bm_secret_key *sk, uint64_t q, uint32_t t,
                                const uint32_t *msg, const uint64_t *mask, const int8_t *err,
                                size_t count, uint64_t *ct_out) {
    if (!sk || !msg || !mask || !err || !ct_out || q < 2 || t < 2 || t > q) return BM_EINVAL;
    const u32 n = sk->p.n;
    for (size_t i = 0; i < count * n; i++)
        if (mask[i] >= q) return BM_EINVAL;
    for (size_t i = 0; i < count; i++)
        encrypt_one(sk, q, t, msg[i], [&](u32 c) { return mask[i * n + c]; }, err[i], ct_out + i * (n + 1));
    return BM_OK;
}

extern "C" bm_status bm_encrypt_seeded(const bm_secret_key *sk, uint64_t q, uint32_t t, const uint32_t *msg,
                                       size_t count, double sigma, uint64_t seed, uint64_t *ct_out) {
    if (!sk || !msg || !ct_out || q < 2 || t < 2 || t > q || !(sigma > 0.0) || sigma > BM_SIGMA_MAX)
        return BM_EINVAL;
    const u32 n = sk->p.n;
    rng::Cdt cdt;
    rng::make_cdt(sigma, cdt);
    for (size_t i = 0; i < count; i++) {
        const int e = rng::gaussian(rng::element(seed, rng::kEncErr, 0, i), cdt);
        encrypt_one(sk, q, t, msg[i],
                    [&](u32 c) { return rng::uniform_mod(rng::element(seed, rng::kEncMask, 0, (uint64_t)i * n + c), q); },
                    e, ct_out + i * (n + 1));
    }
    return BM_OK;
}

extern "C" bm_status bm_decrypt(const bm_secret_key *sk, uint64_t q, uint32_t t,
                                const uint64_t *ct, size_t count, uint32_t *msg_out) {
    if (!sk || !ct || !msg_out || q < 2 || t < 2) return BM_EINVAL;
    const u32 n = sk->p.n;
    for (size_t i = 0; i < count; i++) {
        const u64 *c = ct + i * (n + 1);
        u128 pos = c[n] % q, neg = 0;
        for (u32 k = 0; k < n; k++) {
            if (sk->s[k] > 0) neg += c[k] % q;
            else if (sk->s[k] < 0) pos += c[k] % q;
        }
        const u64 pm = (u64)(pos % q), nm = (u64)(neg % q);
        const u64 ph = pm >= nm ? pm - nm : pm + q - nm;
        msg_out[i] = (uint32_t)((((u128)ph * t + q / 2) / q) % t);
    }
    return BM_OK;
}

extern "C" const char *bm_status_str(bm_status s) {
    switch (s) {
        case BM_OK: return "ok";
        case BM_EINVAL: return "invalid argument";
        case BM_ENOTPRIME: return "modulus is not an NTT-friendly prime";
        case BM_ENOMEM: return "out of device memory";
        case BM_ENONNEGACYCLIC: return "look-up table is not negacyclic";
        case BM_ETIMEDOUT: return "bounded device wait expired";
        case BM_ECUDA: return "CUDA runtime error";
        case BM_EBUSY: return "admission refused";
        case BM_EWORKSPACE: return "workspace too small";
        default: return "unknown status";
    }
}
