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
    if (p->N < 256 || p->N > 4096 || (p->N & (p->N - 1))) return BM_EINVAL;
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

// One RGSW row per block (see the file header for the formula).
__global__ void k_bsk_rows(const u64 *__restrict__ mask, const int8_t *__restrict__ err,
                           const int8_t *__restrict__ s, const u64 *__restrict__ zhat,
                           u64 *__restrict__ bsk, KeyDev K) {
    extern __shared__ u64 sm[];
    const u32 N = K.N, lB = K.l_B;
    const u64 Q = K.mq.Q;
    const size_t row_id = blockIdx.x;
    const u64 *a = mask + row_id * N;
    const int8_t *e = err + row_id * N;
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
        sm[i] = a[i];
        int v = e[i];
        sm[N + i] = v >= 0 ? (u64)v : Q - (u64)(-v);
    }
    __syncthreads();
    cta_ntt_fwd(sm, 2, K.logN, K.tw, K.twsh, Q);
    const u32 row = (u32)(row_id % (2 * lB));
    const u32 sgn = (u32)((row_id / (2 * lB)) % 2);
    const u32 k = (u32)(row_id / (4 * lB));
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
        // stored split into the multiply-accumulate's limbs (KeyDev::lbits)
        const u64 lmask = (1ull << K.lbits) - 1;
        const u64 w0 = mul_shoup(c0, K.ninv, K.ninv_sh, Q), w1 = mul_shoup(c1, K.ninv, K.ninv_sh, Q);
        o[i] = (w0 & lmask) | ((w0 >> K.lbits) << 32);
        o[N + i] = (w1 & lmask) | ((w1 >> K.lbits) << 32);
    }
}

struct KsGadget { u64 g[16]; };

// One key-switching row per warp: (a', <a', s> + e + v z_i g_j).
// mask holds rows [row0, row_end) only; err and ksk are indexed absolutely.
__global__ void k_ksk_rows(const u64 *__restrict__ mask, const int8_t *__restrict__ err,
                           const int8_t *__restrict__ s, const int8_t *__restrict__ z,
                           u64 *__restrict__ ksk, KeyDev K, KsGadget G, size_t row0,
                           size_t row_end) {
    const size_t warp = row0 + (size_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const u32 lane = threadIdx.x & 31;
    if (warp >= row_end) return;
    const u32 n = K.n, B1 = (1u << K.log2_Bks) - 1;
    const u64 Q = K.mq.Q;
    const u64 *a = mask + (warp - row0) * n;
    u64 *o = ksk + warp * (n + 1);
    u64 lo = 0, hi = 0;
    for (u32 c = lane; c < n; c += 32) {
        const u64 x = a[c];
        o[c] = x;
        const int sc = s[c];
        if (sc > 0) add128(lo, hi, x);
        else if (sc < 0) add128(lo, hi, Q - x);
    }
    u64 acc = reduce128(lo, hi, K.mq);
    for (int off = 16; off; off >>= 1) acc = add_mod(acc, __shfl_down_sync(0xffffffffu, acc, off), Q);
    if (lane == 0) {
        const u32 v = (u32)(warp % B1) + 1;
        const u32 j = (u32)((warp / B1) % K.l_ks);
        const u32 i = (u32)(warp / ((size_t)B1 * K.l_ks));
        u64 l2 = 0, h2 = 0;
        mac128(l2, h2, v, G.g[j]);
        u64 vg = reduce128(l2, h2, K.mq);
        const int zi = z[i];
        u64 msg = zi > 0 ? vg : (zi < 0 ? (vg ? Q - vg : 0) : 0);
        const int ev = err[warp];
        const u64 e = ev >= 0 ? (u64)ev : Q - (u64)(-ev);
        o[n] = add_mod(add_mod(acc, e, Q), msg, Q);
    }
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

static bm_status keygen_impl(const bm_key_params *params, const bm_key_randomness *rnd,
                             bm_eval_key *ek) {
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
    BM_CUDA_TRY(cudaMemcpy(d_s.p, rnd->s, n, cudaMemcpyHostToDevice));
    BM_CUDA_TRY(cudaMemcpy(d_z.p, rnd->z, N, cudaMemcpyHostToDevice));

    const u32 threads = N / 2 < 512 ? N / 2 : 512;
    k_ntt_z<<<1, threads, N * 8>>>((const int8_t *)d_z.p, d_zhat, K);
    BM_CUDA_TRY(cudaGetLastError());

    // Bootstrapping keys, in chunks of key indices to bound staging memory.
    {
        const size_t rows_per_k = 2 * 2 * (size_t)lB;
        const u32 kchunk = 64;
        DevBuf d_mask, d_err;
        BM_CUDA_TRY(cudaMalloc(&d_mask.p, kchunk * rows_per_k * N * 8));
        BM_CUDA_TRY(cudaMalloc(&d_err.p, kchunk * rows_per_k * N));
        BM_CUDA_TRY(cudaFuncSetAttribute(k_bsk_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         2 * N * 8));
        for (u32 k0 = 0; k0 < n; k0 += kchunk) {
            const u32 k1 = k0 + kchunk < n ? k0 + kchunk : n;
            const size_t rows = (size_t)(k1 - k0) * rows_per_k;
            BM_CUDA_TRY(cudaMemcpy(d_mask.p, rnd->bsk_mask + (size_t)k0 * rows_per_k * N,
                                   rows * N * 8, cudaMemcpyHostToDevice));
            BM_CUDA_TRY(cudaMemcpy(d_err.p, rnd->bsk_err + (size_t)k0 * rows_per_k * N, rows * N,
                                   cudaMemcpyHostToDevice));
            // the kernel derives k from the row id, so offset the secret
            k_bsk_rows<<<(unsigned)rows, threads, 2 * N * 8>>>(
                (const u64 *)d_mask.p, (const int8_t *)d_err.p, (const int8_t *)d_s.p + k0, d_zhat,
                ek->d_bsk + (size_t)k0 * rows_per_k * 2 * N, K);
            BM_CUDA_TRY(cudaGetLastError());
            BM_CUDA_TRY(cudaDeviceSynchronize());
        }
    }
    // Key-switching keys.
    {
        KsGadget G;
        memset(&G, 0, sizeof(G));
        const u128 P = (u128)1 << (p.log2_Bks * p.l_ks);
        for (u32 j = 0; j < p.l_ks && j < 16; j++)
            G.g[j] = (u64)((((u128)Q << (p.log2_Bks * j)) + P / 2) / P);
        const size_t chunk_rows = 1u << 16;
        DevBuf d_mask, d_err;
        BM_CUDA_TRY(cudaMalloc(&d_mask.p, chunk_rows * n * 8));
        BM_CUDA_TRY(cudaMalloc(&d_err.p, ksk_rows));
        BM_CUDA_TRY(cudaMemcpy(d_err.p, rnd->ksk_err, ksk_rows, cudaMemcpyHostToDevice));
        for (size_t r0 = 0; r0 < ksk_rows; r0 += chunk_rows) {
            const size_t r1 = r0 + chunk_rows < ksk_rows ? r0 + chunk_rows : ksk_rows;
            BM_CUDA_TRY(cudaMemcpy(d_mask.p, rnd->ksk_mask + r0 * n, (r1 - r0) * n * 8,
                                   cudaMemcpyHostToDevice));
            const size_t rows = r1 - r0;
            const unsigned blocks = (unsigned)((rows + 7) / 8);
            k_ksk_rows<<<blocks, 256>>>((const u64 *)d_mask.p, (const int8_t *)d_err.p,
                                        (const int8_t *)d_s.p, (const int8_t *)d_z.p,
                                        ek->d_ksk, K, G, r0, r1);
            BM_CUDA_TRY(cudaGetLastError());
            BM_CUDA_TRY(cudaDeviceSynchronize());
        }
    }
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
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return BM_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return BM_EINVAL;
    bm_eval_key *ek = new (std::nothrow) bm_eval_key();
    if (!ek) return BM_ENOMEM;
    ek->device = device;
    ek->p = *params;
    st = keygen_impl(params, rnd, ek);
    cudaSetDevice(prev);
    if (st != BM_OK) {
        bm_free_eval_key(ek);
        return st;
    }
    bm_secret_key *sk = new (std::nothrow) bm_secret_key();
    sk->p = *params;
    sk->s = (int8_t *)malloc(params->n);
    sk->z = (int8_t *)malloc(params->N);
    memcpy(sk->s, rnd->s, params->n);
    memcpy(sk->z, rnd->z, params->N);
    *sk_out = sk;
    *ek_out = ek;
    return BM_OK;
}

// ---------------------------------------------------------------------------
// Client-side LWE encryption / decryption (Section 2 item (8))
// ---------------------------------------------------------------------------

extern "C" bm_status bm_encrypt(const bm_secret_key *sk, uint64_t q, uint32_t t,
                                const uint32_t *msg, const uint64_t *mask, const int8_t *err,
                                size_t count, uint64_t *ct_out) {
    if (!sk || !msg || !mask || !err || !ct_out || q < 2 || t < 2 || t > q) return BM_EINVAL;
    const u32 n = sk->p.n;
    const u64 delta = q / t;
    for (size_t i = 0; i < count; i++) {
        u64 *o = ct_out + i * (n + 1);
        u128 pos = 0, neg = 0;
        for (u32 c = 0; c < n; c++) {
            const u64 a = mask[i * n + c];
            if (a >= q) return BM_EINVAL;
            o[c] = a;
            if (sk->s[c] > 0) pos += a;
            else if (sk->s[c] < 0) neg += a;
        }
        const int e = err[i];
        pos += (u128)(msg[i] % t) * delta + (e >= 0 ? (u64)e : 0);
        neg += e < 0 ? (u64)(-e) : 0;
        const u64 pm = (u64)(pos % q), nm = (u64)(neg % q);
        o[n] = pm >= nm ? pm - nm : pm + q - nm;
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
