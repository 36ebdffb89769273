// Blind rotation, sample extraction and key switching of BootMMPM
// (arXiv 2310.12441, Algorithm 1) and the C-ABI entry points that launch them.
//
// One thread block runs one job.  Its RLWE-vector accumulator ACC
// ([m][2][N] words, Section 4) lives in two global buffers of the
// workspace (read the old one, write the new one, swap), which stay in L2.
// Per CMux step k (Eq. (cmux:BP)) and per row r the block
//   1. forms D = P(c) ACC - ACC for row r, c = -a_k (sign +) and c = a_k
//      (sign -), reading the source row and monomial of Eq. (ex1:BPc);
//   2. splits each component of D into l_B unsigned base-B digit polynomials
//      (Section 2 item (10)) and transforms them (negacyclic NTT);
//   3. multiplies them with the NTT-domain key rows of ct_k+ / ct_k- and
//      sums all 2 x 2 l_B products per output column in exact 128-bit
//      registers (Section 2 item (14), summed over both CMux terms);
//   4. reduces, inverse-transforms (N^-1 is folded into the key) and adds
//      the result to row r of ACC.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "ntt.cuh"
#include "ntt_reg.cuh"

#include "br_launch.cuh"

// ---------------------------------------------------------------------------
// Sample extraction + key switching
// ---------------------------------------------------------------------------

// a~ = floor((a P + floor(Q/2)) / Q) mod P, exact: the Shoup-style quotient
// estimate floor(a P' / 2^64), P' = floor(P 2^64 / Q), is at most 2 below the
// true quotient; the remainder fits in 64 bits and fixes it.
__device__ __forceinline__ u64 ks_round(u64 a, const KeyDev &K) {
    const u32 sh = K.log2_Bks * K.l_ks;
    const u64 Q = K.mq.Q;
    u64 q = __umul64hi(a, K.ks_pq);
    u64 r = (a << sh) + Q / 2 - q * Q;
    for (int it = 0; it < 3 && r >= Q; it++) { r -= Q; q++; }
    return q & ((1ull << sh) - 1);
}

// Address of `p` (this block's shared memory) in the shared memory of block
// `rank` of the cluster (distributed shared memory), and a load from it.
__device__ __forceinline__ u64 ld_peer_smem(const u64 *p, u32 rank) {
    const u32 local = (u32)__cvta_generic_to_shared(p);
    u32 remote;
    u64 v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(remote) : "memory");
    return v;
}

// Key switching (Eq. (equ-key-swi)) of the LWE_{N,Q} sample given by
// get_a(i) (i < N) and b: out = (0^n, b) - sum_{i,j} KSK(i, j, d_ij).
// The S blocks of a thread-block cluster split the coefficients i (block
// `rank` takes the rank-th slice of N/S); each thread owns columns
// c = tid + q blockDim (q < CPT) and keeps four key rows' loads in flight;
// block 0 then adds the partial sums it reads from its peers' shared memory
// and writes the output.  Shared memory: digits (one byte each) of the
// block's slice, then its n + 1 partial sums.
template <int CPT, typename GetA>
__device__ void key_switch_block(const KeyDev &K, GetA get_a, u64 b, u64 *__restrict__ out, u32 rank, u32 S) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const u32 N = K.N, n = K.n, lks = K.l_ks, B1 = (1u << K.log2_Bks) - 1;
    const u32 i0 = rank * (N / S), i1 = i0 + N / S;
    u64 *part = (u64 *)(dsm + (((size_t)(N / S) * lks + 15) & ~(size_t)15));
    for (u32 i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const u64 at = ks_round(get_a(i), K);
        for (u32 j = 0; j < lks; j++)
            dsm[(i - i0) * lks + j] = (unsigned char)((at >> (K.log2_Bks * j)) & B1);
    }
    __syncthreads();
    u64 lo[CPT], hi[CPT];
#pragma unroll
    for (int q = 0; q < CPT; q++) lo[q] = hi[q] = 0;
    const size_t rowlen = n + 1;
    const u32 rows = (i1 - i0) * lks;
    constexpr int KR = CPT == 4 ? 4 : 2;
    for (u32 r0 = 0; r0 < rows; r0 += KR) {
        const u64 *rp[KR];
        bool ok[KR];
#pragma unroll
        for (int k = 0; k < KR; k++) {
            const u32 rr = r0 + k;
            const u32 d = rr < rows ? dsm[rr] : 0;    // digit d_ij of row rr = (i - i0) lks + j
            ok[k] = d != 0;
            const u32 i = i0 + rr / lks, j = rr % lks;
            rp[k] = K.ksk + (((size_t)i * lks + j) * B1 + (ok[k] ? d - 1 : 0)) * rowlen;
        }
        u64 v[KR][CPT];
#pragma unroll
        for (int k = 0; k < KR; k++)
#pragma unroll
            for (int q = 0; q < CPT; q++) {
                const u32 c = threadIdx.x + q * blockDim.x;
                v[k][q] = (ok[k] && c <= n) ? __ldg(rp[k] + c) : 0;
            }
#pragma unroll
        for (int k = 0; k < KR; k++)
#pragma unroll
            for (int q = 0; q < CPT; q++) add128(lo[q], hi[q], v[k][q]);
    }
    const u64 Q = K.mq.Q;
#pragma unroll
    for (int q = 0; q < CPT; q++) {
        const u32 c = threadIdx.x + q * blockDim.x;
        if (c <= n) part[c] = reduce128(lo[q], hi[q], K.mq);
    }
    if (S > 1) cluster_sync(); else __syncthreads();
    if (rank == 0) {
        for (u32 c = threadIdx.x; c <= n; c += blockDim.x) {
            u64 sum = part[c];
            for (u32 r = 1; r < S; r++) sum = add_mod(sum, ld_peer_smem(part + c, r), Q);
            out[c] = sub_mod(c == n ? b : 0, sum, Q);
        }
    }
    // peers keep their shared memory until block 0 has read it
    if (S > 1) cluster_sync();
}

// Row 0 of the final ACC -> LWE_{N,Q} (Eq. (equ-sam-extr)) -> key switch;
// a cluster of S blocks per job (S = 1: plain launch, one block per job).
// Launch bounds: 256 threads with 4 columns each (n < 1024), else up to 640
// threads with 8 columns each (n < 5120).
#define BM_KS_BOUNDS(CPT) __launch_bounds__((CPT) == 4 ? 256 : 640)

template <int CPT>
__global__ void BM_KS_BOUNDS(CPT) k_extract_keyswitch(const DevJob *__restrict__ jobs, u32 steps_limit,
                                    const u64 *__restrict__ ws, u64 *__restrict__ ct_out) {
    const u32 S = cluster_size(), rank = cluster_rank();
    const DevJob J = jobs[blockIdx.x / S];
    const KeyDev &K = *J.key;
    const u32 N = K.N;
    const u32 steps = steps_limit < K.n ? steps_limit : K.n;
    const u64 *acc = ws + J.acc_off + ((steps & 1) ? (size_t)J.m * 2 * N : 0);
    const u64 Q = K.mq.Q;
    auto get_a = [&](u32 i) -> u64 {
        if (i == 0) return acc[0];
        const u64 v = acc[N - i];
        return v ? Q - v : 0;
    };
    key_switch_block<CPT>(K, get_a, acc[N], ct_out + J.out_off, rank, S);
}

template <int CPT>
__global__ void BM_KS_BOUNDS(CPT) k_key_switch(const KeyDev *Kp, const u64 *__restrict__ lwe_in, u64 *__restrict__ out) {
    const KeyDev &K = *Kp;
    const u32 S = cluster_size(), rank = cluster_rank();
    const size_t job = blockIdx.x / S;
    const u64 *in = lwe_in + job * (K.N + 1);
    auto get_a = [&](u32 i) -> u64 { return in[i]; };
    key_switch_block<CPT>(K, get_a, in[K.N], out + job * (K.n + 1), rank, S);
}

__global__ void k_sample_extract(const KeyDev *Kp, const u64 *__restrict__ rlwe, u64 *__restrict__ lwe) {
    const KeyDev &K = *Kp;
    const u32 N = K.N;
    const u64 Q = K.mq.Q;
    const u64 *a = rlwe + (size_t)blockIdx.x * 2 * N;
    u64 *o = lwe + (size_t)blockIdx.x * (N + 1);
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
        const u64 v = i == 0 ? a[0] : a[N - i];
        o[i] = (i == 0 || v == 0) ? v : Q - v;
    }
    if (threadIdx.x == 0) o[N] = a[N];
}

__global__ void k_copy_acc(const DevJob *__restrict__ jobs, u32 steps_limit, const u64 *__restrict__ ws,
                           u64 *__restrict__ out) {
    const DevJob J = jobs[blockIdx.x];
    const u32 N = J.N;
    const u32 steps = steps_limit < J.n ? steps_limit : J.n;
    const size_t words = (size_t)J.m * 2 * N;
    const u64 *acc = ws + J.acc_off + ((steps & 1) ? words : 0);
    for (size_t i = threadIdx.x; i < words; i += blockDim.x) out[J.out_off + i] = acc[i];
}

// Negacyclic products through the NTT: one pair per block.
__global__ void k_poly_mul(const KeyDev *Kp, const u64 *__restrict__ a, const u64 *__restrict__ b,
                           u64 *__restrict__ out) {
    extern __shared__ u64 sm[];
    const KeyDev &K = *Kp;
    const u32 N = K.N;
    const u64 Q = K.mq.Q;
    const size_t off = (size_t)blockIdx.x * N;
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
        sm[i] = a[off + i] % Q;
        sm[N + i] = b[off + i] % Q;
    }
    __syncthreads();
    cta_ntt_fwd(sm, 2, K.logN, K.tw, K.twsh, Q);
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
        u64 lo = 0, hi = 0;
        mac128(lo, hi, sm[i], sm[N + i]);
        sm[i] = mul_shoup(reduce128(lo, hi, K.mq), K.ninv, K.ninv_sh, Q);
    }
    __syncthreads();
    cta_ntt_inv(sm, 1, K.logN, K.itw, K.itwsh, Q);
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) out[off + i] = sm[i];
}

// Modulus switch (Section 2 (9)) of every word: round half up.
__global__ void k_mod_switch(const u64 *__restrict__ in, u64 *__restrict__ out, size_t words, u64 q_from,
                             u64 q_to) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (size_t)gridDim.x * blockDim.x) {
        const unsigned __int128 x = (unsigned __int128)(in[i] % q_from) * q_to + q_from / 2;
        out[i] = (u64)((x / q_from) % q_to);
    }
}

// Tables of the two-round method over Z_{2t} (see bm_bootstrap_arbitrary):
// mp (shared by all jobs) and, per job, the negacyclic extension F of f.
__global__ void k_two_round_tables(const u32 *__restrict__ f, u32 t, u32 count, u32 *__restrict__ mp,
                                   u32 *__restrict__ F) {
    const u32 T = 2 * t;
    const size_t total = (size_t)count * T;
    for (size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x; w < total + T;
         w += (size_t)gridDim.x * blockDim.x) {
        if (w < T) {
            const u32 x = (u32)w;
            mp[x] = (x < t / 2 || x >= 3 * t / 2) ? T - t / 2 : t / 2;
            continue;
        }
        const size_t j = (w - T) / T;
        const u32 y = (u32)((w - T) % T);
        const u32 *fj = f + j * t;
        u32 v;
        if (y < t / 2) v = fj[y] % T;
        else if (y >= 3 * t / 2) v = fj[y - t] % T;
        else {
            const u32 z = (y + t) % T;    // (y - t) mod 2t, in [0, t/2) or [3t/2, 2t)
            const u32 fz = z < t / 2 ? fj[z] : fj[z - t];
            v = (T - fz % T) % T;
        }
        F[j * T + y] = v;
    }
}

// out = x - y mod q word by word, and add_b added to the last word (b) of
// every ciphertext of n + 1 words.
__global__ void k_lwe_sub(const u64 *__restrict__ x, const u64 *__restrict__ y, u64 *__restrict__ out,
                          size_t count, u32 n, u64 q, u64 add_b) {
    const size_t words = count * (n + 1);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (size_t)gridDim.x * blockDim.x) {
        u64 v = sub_mod(x[i] % q, y[i] % q, q);
        if (i % (n + 1) == n) v = add_mod(v, add_b, q);
        out[i] = v;
    }
}

// Throughput probe of the blind rotation's own modular product: the
// three-product Shoup multiplication for Q = c 2^32 + 1 (shoup3_qlow1_lazy:
// seven multiplier instructions, 22 multiplier-pipe cycles per warp), eight
// independent chains per thread; every output in [0, 4Q) is a valid next
// input.
__global__ void k_modmul_probe(u64 *out, u32 iters, u32 c, u64 w, u64 wsh) {
    u64 x0 = threadIdx.x + 1, x1 = x0 + 7, x2 = x0 + 13, x3 = x0 + 29;
    u64 x4 = x0 + 31, x5 = x0 + 37, x6 = x0 + 41, x7 = x0 + 43;
    for (u32 i = 0; i < iters; i++) {
        x0 = shoup3_qlow1_lazy(x0, w, wsh, c);
        x1 = shoup3_qlow1_lazy(x1, w, wsh, c);
        x2 = shoup3_qlow1_lazy(x2, w, wsh, c);
        x3 = shoup3_qlow1_lazy(x3, w, wsh, c);
        x4 = shoup3_qlow1_lazy(x4, w, wsh, c);
        x5 = shoup3_qlow1_lazy(x5, w, wsh, c);
        x6 = shoup3_qlow1_lazy(x6, w, wsh, c);
        x7 = shoup3_qlow1_lazy(x7, w, wsh, c);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 ^ x1 ^ x2 ^ x3 ^ x4 ^ x5 ^ x6 ^ x7;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// A run of plan jobs [first, last) with one ring degree and variant, run by
// one persistent kernel.
struct ClassRange {
    uint32_t first, last;
    u32 N, variant;
};

struct Plan {
    size_t jobs_off, acc_off_bytes, total;
    std::vector<DevJob> dj;
    std::vector<ClassRange> classes;   // persistent classes (order_by_cost plans)
    std::vector<u32> gen;     // prefix sums of the jobs' generators, uploaded after the job table
};

// The generator exponents of job i: gens + gen_off[i] (m words), or none
// (gens == nullptr or gen_off[i] == BM_GEN_EXAMPLE1) for Example 1's P(1).
const uint32_t *job_gen(const uint32_t *gens, const uint64_t *gen_off, uint32_t i) {
    if (!gens || !gen_off || gen_off[i] == BM_GEN_EXAMPLE1) return nullptr;
    return gens + gen_off[i];
}

// Theorem 1: the action is transitive iff ord(x^{sum u}) = 2N, i.e. sum u odd.
bm_status validate_gens(const bm_eval_key *const *keys, const bm_job *jobs, uint32_t count,
                        const uint32_t *gens, const uint64_t *gen_off) {
    if (!gens) return BM_OK;
    if (!gen_off) return BM_EINVAL;
    for (uint32_t i = 0; i < count; i++) {
        const uint32_t *u = job_gen(gens, gen_off, i);
        if (!u) continue;
        const u32 twoN = 2 * keys[jobs[i].key]->p.N;
        u64 S = 0;
        for (u32 k = 0; k < jobs[i].m; k++) {
            if (u[k] >= twoN) return BM_EINVAL;
            S += u[k];
        }
        if (!(S & 1)) return BM_EINVAL;
    }
    return BM_OK;
}

bm_status validate_jobs(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                        uint32_t count, int *device) {
    if (!keys || n_keys == 0 || (!jobs && count)) return BM_EINVAL;
    for (uint32_t i = 0; i < n_keys; i++)
        if (!keys[i]) return BM_EINVAL;
    *device = keys[0]->device;
    for (uint32_t i = 0; i < n_keys; i++)
        if (keys[i]->device != *device) return BM_EINVAL;
    for (uint32_t i = 0; i < count; i++) {
        const bm_job &j = jobs[i];
        if (j.key >= n_keys || j.reserved) return BM_EINVAL;
        const bm_eval_key *k = keys[j.key];
        if (j.m < 1 || j.m > BM_MAX_M || 2ull * k->p.N * j.m > BM_MAX_QP) return BM_EINVAL;
        if (k->p.N > BM_MAX_N_BLOCK && j.m != 1) return BM_EINVAL;   // big.cu: the single-polynomial layout
        if (j.t < 2 || (j.t & 1) || (u64)j.t > 2ull * k->p.N * j.m) return BM_EINVAL;
    }
    return BM_OK;
}

// Work of one job in butterfly units (n m N log2 N), for longest-first order.
double job_cost(const DevJob &d) {
    double lg = 0;
    while ((1u << (u32)lg) < d.N) lg += 1;
    return (double)d.n * d.m * d.N * lg;
}

// The device job table is reordered (outputs still go to the jobs' own
// offsets): by ring degree and variant for one-block-per-job launches, or,
// with order_by_cost, longest first for the persistent kernel.
bm_status make_plan(const bm_eval_key *const *keys, const bm_job *jobs, uint32_t count, Plan &pl,
                    bool order_by_cost = false, const uint32_t *gens = nullptr,
                    const uint64_t *gen_off = nullptr) {
    pl.jobs_off = BM_WS_HEADER;
    // prefix sums of the generators right after the job table (one upload)
    const size_t gen_base = pl.jobs_off + sizeof(DevJob) * (size_t)count;   // bytes, 8-aligned
    pl.gen.clear();
    for (uint32_t i = 0; i < count; i++) {
        const uint32_t *u = job_gen(gens, gen_off, i);
        if (u) pl.gen.resize(pl.gen.size() + jobs[i].m + 1);
    }
    size_t off = align_up(gen_base + 4 * pl.gen.size(), 256);
    pl.acc_off_bytes = off;
    pl.dj.resize(count);
    size_t gpos = 0;
    size_t acc_words = 0;
    for (uint32_t i = 0; i < count; i++) {
        const bm_eval_key *k = keys[jobs[i].key];
        DevJob &d = pl.dj[i];
        d.key = k->d_view;
        d.m = jobs[i].m;
        d.t = jobs[i].t;
        d.N = k->p.N;
        d.n = k->p.n;
        d.in_off = jobs[i].in_off;
        d.lut_off = jobs[i].lut_off;
        d.out_off = jobs[i].out_off;
        d.acc_off = acc_words;
        d.variant = choose_variant(k->p);
        limb_plan(k->p, d.variant, d.lbits, d.fold_each);   // lbits as in the key's BSK
        d.pad = 0;
        d.gS = d.gSinv = 0;
        d.gpre = 0;
        if (const uint32_t *u = job_gen(gens, gen_off, i)) {
            const u32 twoN = 2 * k->p.N, m = jobs[i].m;
            u32 *pre = pl.gen.data() + gpos;
            pre[0] = 0;
            for (u32 q = 0; q < m; q++) pre[q + 1] = (pre[q] + u[q]) % twoN;
            d.gS = pre[m];
            u32 inv = 1;   // S^-1 mod 2N (S odd; 2N a power of two): Newton's iteration
            for (int it = 0; it < 6; it++) inv = inv * (2u - d.gS * inv);
            d.gSinv = inv % twoN;
            d.gpre = (gen_base + 4 * gpos) / 4;
            gpos += m + 1;
        }
        acc_words += 3ull * 2 * jobs[i].m * k->p.N + bm_big_extra_words(k->p.N, k->p.l_B);
    }
    pl.classes.clear();
    if (order_by_cost) {
        // jobs of ring degree 1024..4096 first (the persistent kernels'
        // share), grouped into classes of equal degree and variant, the class
        // with the longest job first and every class longest job first; the
        // rest grouped by degree and variant
        auto eligible = [](const DevJob &d) { return d.N >= 1024 && d.N <= 4096; };
        auto key = [](const DevJob &d) { return ((u64)d.N << 32) | d.variant; };
        std::vector<std::pair<u64, double>> top;   // class key -> its longest job
        for (const DevJob &d : pl.dj) {
            if (!eligible(d)) continue;
            bool found = false;
            for (auto &kv : top)
                if (kv.first == key(d)) {
                    kv.second = std::max(kv.second, job_cost(d));
                    found = true;
                }
            if (!found) top.push_back({key(d), job_cost(d)});
        }
        auto rank = [&](const DevJob &d) {
            double c = 0;
            for (auto &kv : top)
                if (kv.first == key(d)) c = kv.second;
            return c;
        };
        std::stable_sort(pl.dj.begin(), pl.dj.end(), [&](const DevJob &a, const DevJob &b) {
            const bool pa = eligible(a), pb = eligible(b);
            if (pa != pb) return pa;
            if (pa) {
                if (key(a) != key(b)) {
                    const double ra = rank(a), rb = rank(b);
                    return ra != rb ? ra > rb : key(a) < key(b);
                }
                return job_cost(a) > job_cost(b);
            }
            return a.N != b.N ? a.N < b.N : a.variant < b.variant;
        });
        for (uint32_t i = 0; i < count && eligible(pl.dj[i]); i++) {
            if (pl.classes.empty() || key(pl.dj[i]) != key(pl.dj[pl.classes.back().first]))
                pl.classes.push_back({i, i + 1, pl.dj[i].N, pl.dj[i].variant});
            else
                pl.classes.back().last = i + 1;
        }
    } else {
        // one launch per run of equal degree and variant: group them
        std::stable_sort(pl.dj.begin(), pl.dj.end(), [](const DevJob &a, const DevJob &b) {
            return a.N != b.N ? a.N < b.N : a.variant < b.variant;
        });
    }
    pl.total = off + acc_words * 8;
    return BM_OK;
}

// Kernel shape per ring degree (log2 N = 8..13) used by launches that do
// not carry their own: the autotuner's choice once it has run, else the
// measured best of each degree (radix 8 with 1024 threads for N = 1024 ..
// 8192; radix 16 with 512 threads below).
constexpr u32 kDefaultShape[14] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1};
std::atomic<u32> g_shape[14] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1};

struct Shapes {
    u32 s[14];
    static Shapes current() {
        Shapes x;
        for (int i = 0; i < 14; i++) x.s[i] = g_shape[i].load();
        return x;
    }
};

u32 log2u(u32 N) {
    u32 l = 0;
    while ((1u << l) < N) l++;
    return l;
}

bm_status launch_br_any(u32 N, u32 variant, u32 shape, const DevJob *jobs, uint32_t cnt, u32 mmax, u32 max_cluster,
                    u32 steps, const uint64_t *ct_in, const uint32_t *lut, u64 *ws_acc, u32 *status,
                    cudaStream_t st, bool dry) {
    switch (N) {
        case 256:
        case 512:
            return bm_launch_br_small(N, variant, shape, jobs, cnt, mmax, max_cluster, steps, ct_in, lut, ws_acc,
                                      status, st, dry);
        case 1024:
            return bm_launch_br_n1024(variant, shape, jobs, cnt, mmax, max_cluster, steps, ct_in, lut, ws_acc,
                                      status, st, dry);
        case 2048:
            return bm_launch_br_n2048(variant, shape, jobs, cnt, mmax, max_cluster, steps, ct_in, lut, ws_acc,
                                      status, st, dry);
        case 4096:
            return bm_launch_br_n4096(variant, shape, jobs, cnt, mmax, max_cluster, steps, ct_in, lut, ws_acc,
                                      status, st, dry);
        case 8192:
            return bm_launch_br_n8192(variant, shape, jobs, cnt, mmax, max_cluster, steps, ct_in, lut, ws_acc,
                                      status, st, dry);
        default: return BM_EINVAL;
    }
}

// Blind rotation of jobs [first, last) of the plan, one launch per run of
// equal ring degree and variant; each job takes one block, or a cluster of up
// to max_cluster blocks when the run has fewer jobs than the GPU has room for.
bm_status run_groups(const Plan &pl, uint32_t first, uint32_t last, u32 steps, const uint64_t *d_ct_in,
                     const uint32_t *d_lut, char *ws, cudaStream_t st, bool dry, u32 max_cluster,
                     const Shapes &shapes) {
    const DevJob *d_jobs = (const DevJob *)(ws + pl.jobs_off);
    u64 *ws_acc = (u64 *)(ws + pl.acc_off_bytes);
    u32 *status = (u32 *)ws;
    uint32_t i = first;
    while (i < last) {
        const u32 N = pl.dj[i].N;
        const u32 variant = pl.dj[i].variant;
        u32 mmax = pl.dj[i].m;
        uint32_t j = i + 1;
        while (j < last && pl.dj[j].N == N && pl.dj[j].variant == variant) {
            mmax = pl.dj[j].m > mmax ? pl.dj[j].m : mmax;
            j++;
        }
        bm_status s;
        if (N > BM_MAX_N_BLOCK) {
            // the launch covers the most steps any of its keys has
            u32 nmax = 0;
            for (uint32_t q = i; q < j; q++) nmax = pl.dj[q].n > nmax ? pl.dj[q].n : nmax;
            s = dry ? BM_OK
                    : bm_launch_br_big(N, d_jobs + i, j - i, steps < nmax ? steps : nmax, d_ct_in, d_lut, ws_acc,
                                       status, st);
        } else {
            s = launch_br_any(N, variant, shapes.s[log2u(N)], d_jobs + i, j - i, mmax, max_cluster, steps, d_ct_in,
                              d_lut, ws_acc, status, st, dry);
        }
        if (s != BM_OK) return s;
        i = j;
    }
    return BM_OK;
}

// Number of leading plan jobs that the persistent kernels handle (ring
// degree 1024..4096); make_plan(order_by_cost) puts them first.
uint32_t persistent_prefix(const Plan &pl) {
    return pl.classes.empty() ? 0 : pl.classes.back().last;
}

// Side streams and events that run persistent classes concurrently.
struct Fork {
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;      // [0] fork, [1 + c] join of side stream c
};

struct KsShape {
    u32 threads, cpt;
    size_t smem;   // digits of all N coefficients (one block per job) + partial sums
    u32 maxN, maxlks, maxn;
    // shared memory when S blocks split a job's coefficients
    size_t smem_for(u32 S) const { return align_up((size_t)(maxN / S) * maxlks, 16) + 8 * (size_t)(maxn + 1); }
};

KsShape ks_shape(const bm_eval_key *const *keys, uint32_t n_keys) {
    u32 maxN = 0, maxn = 0, maxlks = 0;
    for (uint32_t i = 0; i < n_keys; i++) {
        maxN = keys[i]->p.N > maxN ? keys[i]->p.N : maxN;
        maxn = keys[i]->p.n > maxn ? keys[i]->p.n : maxn;
        maxlks = keys[i]->p.l_ks > maxlks ? keys[i]->p.l_ks : maxlks;
    }
    KsShape k;
    k.cpt = maxn + 1 <= 1024 ? 4 : 8;
    k.threads = k.cpt == 4 ? 256 : ((maxn + 1 + 7) / 8 + 31) / 32 * 32;
    k.maxN = maxN;
    k.maxlks = maxlks;
    k.maxn = maxn;
    k.smem = k.smem_for(1);
    return k;
}

// Blocks per job of the key switch: the largest S in {1, 2, 4, 8} with
// count S <= SMs (one block per job once the batch fills the GPU).
u32 ks_split(uint32_t count, int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 1;
    u32 S = 1;
    while (S < 8 && (u64)count * (2 * S) <= (u64)sms) S *= 2;
    return S;
}

template <typename Kern, typename... Args>
bm_status launch_ks_kernel(Kern kern, uint32_t count, u32 S, const KsShape &ks, cudaStream_t st, Args... args) {
    static std::atomic<uint64_t> attr_done{0};
    bm_status s = ensure_smem(kern, 96 * 1024, attr_done);
    if (s != BM_OK) return s;
    // large ring degrees (digits of N coefficients above 96 KB) split every
    // job's coefficients over more blocks of a cluster
    while (S < 8 && ks.smem_for(S) > 96 * 1024) S *= 2;
    const size_t smem = ks.smem_for(S);
    if (smem > 96 * 1024) return BM_EINVAL;
    if (S == 1) {
        kern<<<count, ks.threads, smem, st>>>(args...);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(count * S);
        cfg.blockDim = dim3(ks.threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = S;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        BM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, args...));
    }
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

bm_status launch_extract_ks(const KsShape &ks, uint32_t count, u32 S, cudaStream_t st, const DevJob *d_jobs,
                            u32 steps, const u64 *ws_acc, uint64_t *d_out) {
    if (ks.cpt == 4)
        return launch_ks_kernel(k_extract_keyswitch<4>, count, S, ks, st, d_jobs, steps, ws_acc, d_out);
    return launch_ks_kernel(k_extract_keyswitch<8>, count, S, ks, st, d_jobs, steps, ws_acc, d_out);
}

// Every launch of one batch (the plan is already in the workspace).
// Largest thread-block cluster (blocks per job) a grouped launch may use.
constexpr u32 kMaxCluster = 8;

bm_status launch_all(const Plan &pl, uint32_t n_persistent, const KsShape &ks, int device, u32 steps, bool do_ks,
                     const uint64_t *d_ct_in, const uint32_t *d_lut, uint64_t *d_out, char *ws,
                     cudaStream_t st, const Shapes &shapes, u32 max_cluster = kMaxCluster,
                     const Fork *fork = nullptr) {
    const uint32_t count = (uint32_t)pl.dj.size();
    const DevJob *d_jobs = (const DevJob *)(ws + pl.jobs_off);
    u64 *ws_acc = (u64 *)(ws + pl.acc_off_bytes);
    bm_status s;
    if (n_persistent) {
        // class 0 (the longest jobs) on `st`, the others on side streams
        // forked from it, so each later class fills SMs as the earlier ones
        // run out of jobs; all join back into `st` before the key switch
        const size_t nc = pl.classes.size();
        if (nc > 1) BM_CUDA_TRY(cudaEventRecord(fork->ev[0], st));
        for (size_t c = 0; c < nc; c++) {
            const ClassRange &cr = pl.classes[c];
            cudaStream_t cs = c == 0 ? st : fork->side[c - 1];
            if (c > 0) BM_CUDA_TRY(cudaStreamWaitEvent(cs, fork->ev[0], 0));
            s = bm_launch_persistent_class(cr.N, cr.variant, shapes.s[log2u(cr.N)], d_jobs + cr.first,
                                           cr.last - cr.first, steps, d_ct_in, d_lut, ws_acc, (u32 *)ws,
                                           (u32 *)ws + BM_WS_COUNTER_WORD + c, device, false, cs);
            if (s != BM_OK) return s;
            if (c > 0) BM_CUDA_TRY(cudaEventRecord(fork->ev[c], cs));
        }
        for (size_t c = 1; c < nc; c++) BM_CUDA_TRY(cudaStreamWaitEvent(st, fork->ev[c], 0));
    }
    if ((s = run_groups(pl, n_persistent, count, steps, d_ct_in, d_lut, ws, st, false, max_cluster, shapes)) != BM_OK)
        return s;
    if (do_ks) {
        if ((s = launch_extract_ks(ks, count, ks_split(count, device), st, d_jobs, steps, ws_acc, d_out)) != BM_OK)
            return s;
    } else {
        k_copy_acc<<<count, 256, 0, st>>>(d_jobs, steps, ws_acc, d_out);
    }
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

bm_status upload_plan(const Plan &pl, char *ws, cudaStream_t st) {
    if (!pl.dj.empty())
        BM_CUDA_TRY(cudaMemcpyAsync(ws + pl.jobs_off, pl.dj.data(), sizeof(DevJob) * pl.dj.size(),
                                    cudaMemcpyHostToDevice, st));
    if (!pl.gen.empty())
        BM_CUDA_TRY(cudaMemcpyAsync(ws + pl.jobs_off + sizeof(DevJob) * pl.dj.size(), pl.gen.data(),
                                    4 * pl.gen.size(), cudaMemcpyHostToDevice, st));
    return BM_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" size_t bm_workspace_bytes(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                     uint32_t count) {
    int dev = 0;
    if (validate_jobs(keys, n_keys, jobs, count, &dev) != BM_OK) return 0;
    Plan pl;
    make_plan(keys, jobs, count, pl);
    return pl.total;
}

static bm_status bootstrap_impl(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                uint32_t count, u32 steps, bool do_ks, const uint64_t *d_ct_in,
                                const uint32_t *d_lut, uint64_t *d_out, void *d_ws, size_t ws_bytes,
                                void *stream, const uint32_t *gens = nullptr,
                                const uint64_t *gen_off = nullptr) {
    int dev = 0;
    bm_status s = validate_jobs(keys, n_keys, jobs, count, &dev);
    if (s != BM_OK) return s;
    if ((s = validate_gens(keys, jobs, count, gens, gen_off)) != BM_OK) return s;
    if (!d_ws || ((uintptr_t)d_ws & 255)) return BM_EINVAL;
    if (count && (!d_ct_in || !d_lut || !d_out)) return BM_EINVAL;
    Plan pl;
    make_plan(keys, jobs, count, pl, false, gens, gen_off);
    if (ws_bytes < pl.total) return BM_EWORKSPACE;
    if (count == 0) return BM_OK;
    DeviceGuard g(dev);
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    if ((s = upload_plan(pl, ws, st)) != BM_OK) return s;
    return launch_all(pl, 0, ks_shape(keys, n_keys), dev, steps, do_ks, d_ct_in, d_lut, d_out, ws, st,
                      Shapes::current());
}

extern "C" bm_status bm_bootstrap_batch(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                        uint32_t count, const uint64_t *d_ct_in, const uint32_t *d_lut,
                                        uint64_t *d_ct_out, void *d_ws, size_t ws_bytes, void *stream) {
    return bootstrap_impl(keys, n_keys, jobs, count, 0xffffffffu, true, d_ct_in, d_lut, d_ct_out, d_ws,
                          ws_bytes, stream);
}

extern "C" size_t bm_workspace_bytes_gen(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                         uint32_t count, const uint32_t *gens, const uint64_t *gen_off) {
    int dev = 0;
    if (validate_jobs(keys, n_keys, jobs, count, &dev) != BM_OK) return 0;
    if (validate_gens(keys, jobs, count, gens, gen_off) != BM_OK) return 0;
    Plan pl;
    make_plan(keys, jobs, count, pl, false, gens, gen_off);
    return pl.total;
}

extern "C" bm_status bm_bootstrap_batch_gen(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                            uint32_t count, const uint32_t *gens, const uint64_t *gen_off,
                                            const uint64_t *d_ct_in, const uint32_t *d_lut, uint64_t *d_ct_out,
                                            void *d_ws, size_t ws_bytes, void *stream) {
    return bootstrap_impl(keys, n_keys, jobs, count, 0xffffffffu, true, d_ct_in, d_lut, d_ct_out, d_ws,
                          ws_bytes, stream, gens, gen_off);
}

extern "C" bm_status bm_blind_rotate(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                     uint32_t count, uint32_t steps, const uint64_t *d_ct_in,
                                     const uint32_t *d_lut, uint64_t *d_acc_out, void *d_ws, size_t ws_bytes,
                                     void *stream) {
    return bootstrap_impl(keys, n_keys, jobs, count, steps, false, d_ct_in, d_lut, d_acc_out, d_ws,
                          ws_bytes, stream);
}

extern "C" size_t bm_host_staging_bytes(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                        uint32_t count) {
    int dev = 0;
    if (validate_jobs(keys, n_keys, jobs, count, &dev) != BM_OK) return 0;
    size_t in_w = 0, lut_w = 0, out_w = 0;
    for (uint32_t i = 0; i < count; i++) {
        const bm_eval_key *k = keys[jobs[i].key];
        in_w = jobs[i].in_off + k->p.n + 1 > in_w ? jobs[i].in_off + k->p.n + 1 : in_w;
        lut_w = jobs[i].lut_off + jobs[i].t > lut_w ? jobs[i].lut_off + jobs[i].t : lut_w;
        out_w = jobs[i].out_off + k->p.n + 1 > out_w ? jobs[i].out_off + k->p.n + 1 : out_w;
    }
    return align_up(in_w * 8, 256) + align_up(lut_w * 4, 256) + align_up(out_w * 8, 256);
}

extern "C" bm_status bm_bootstrap_batch_host(const bm_eval_key *const *keys, uint32_t n_keys,
                                             const bm_job *jobs, uint32_t count, const uint64_t *h_ct_in,
                                             size_t ct_in_words, const uint32_t *h_lut, size_t lut_words,
                                             uint64_t *h_ct_out, size_t ct_out_words, void *d_ws,
                                             size_t ws_bytes, void *stream) {
    int dev = 0;
    bm_status s = validate_jobs(keys, n_keys, jobs, count, &dev);
    if (s != BM_OK) return s;
    if (!h_ct_in || !h_lut || !h_ct_out || !d_ws) return BM_EINVAL;
    for (uint32_t i = 0; i < count; i++) {
        const bm_eval_key *k = keys[jobs[i].key];
        if (jobs[i].in_off + k->p.n + 1 > ct_in_words || jobs[i].lut_off + jobs[i].t > lut_words ||
            jobs[i].out_off + k->p.n + 1 > ct_out_words)
            return BM_EINVAL;
    }
    const size_t need = bm_workspace_bytes(keys, n_keys, jobs, count);
    const size_t stage = bm_host_staging_bytes(keys, n_keys, jobs, count);
    if (ws_bytes < need + stage) return BM_EWORKSPACE;
    DeviceGuard g(dev);
    cudaStream_t st = (cudaStream_t)stream;
    char *base = (char *)d_ws + align_up(need, 256);
    uint64_t *d_in = (uint64_t *)base;
    uint32_t *d_lut = (uint32_t *)(base + align_up(ct_in_words * 8, 256));
    uint64_t *d_out = (uint64_t *)((char *)d_lut + align_up(lut_words * 4, 256));
    if ((char *)d_out + ct_out_words * 8 > (char *)d_ws + ws_bytes) return BM_EWORKSPACE;
    BM_CUDA_TRY(cudaMemcpyAsync(d_in, h_ct_in, ct_in_words * 8, cudaMemcpyHostToDevice, st));
    BM_CUDA_TRY(cudaMemcpyAsync(d_lut, h_lut, lut_words * 4, cudaMemcpyHostToDevice, st));
    s = bm_bootstrap_batch(keys, n_keys, jobs, count, d_in, d_lut, d_out, d_ws, need, stream);
    if (s != BM_OK) return s;
    BM_CUDA_TRY(cudaMemcpyAsync(h_ct_out, d_out, ct_out_words * 8, cudaMemcpyDeviceToHost, st));
    BM_CUDA_TRY(cudaStreamSynchronize(st));
    return BM_OK;
}

extern "C" bm_status bm_sample_extract(const bm_eval_key *key, const uint64_t *d_rlwe, uint32_t count,
                                       uint64_t *d_lwe_out, void *stream) {
    if (!key || (count && (!d_rlwe || !d_lwe_out))) return BM_EINVAL;
    if (!count) return BM_OK;
    DeviceGuard g(key->device);
    k_sample_extract<<<count, 256, 0, (cudaStream_t)stream>>>(key->d_view, d_rlwe, d_lwe_out);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

extern "C" bm_status bm_key_switch(const bm_eval_key *key, const uint64_t *d_lwe_in, uint32_t count,
                                   uint64_t *d_out, void *stream) {
    if (!key || (count && (!d_lwe_in || !d_out))) return BM_EINVAL;
    if (!count) return BM_OK;
    DeviceGuard g(key->device);
    const bm_eval_key *keys[1] = {key};
    const KsShape ks = ks_shape(keys, 1);
    const u32 S = ks_split(count, key->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ks.cpt == 4) return launch_ks_kernel(k_key_switch<4>, count, S, ks, st, key->d_view, d_lwe_in, d_out);
    return launch_ks_kernel(k_key_switch<8>, count, S, ks, st, key->d_view, d_lwe_in, d_out);
}

extern "C" bm_status bm_poly_mul(const bm_eval_key *key, const uint64_t *d_a, const uint64_t *d_b,
                                 uint32_t count, uint64_t *d_out, void *stream) {
    if (!key || (count && (!d_a || !d_b || !d_out))) return BM_EINVAL;
    if (!count) return BM_OK;
    DeviceGuard g(key->device);
    const u32 N = key->p.N;
    if (N > BM_MAX_N_BLOCK) {
        // two-pass transforms over global memory; scratch for the second operand
        u64 *scratch = nullptr;
        BM_CUDA_TRY(cudaMalloc(&scratch, (size_t)count * N * 8));
        bm_status s = bm_big_poly_mul(d_a, d_b, count, d_out, scratch, key->d_view, key->p.Q, N, (cudaStream_t)stream);
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        cudaFree(scratch);
        if (s != BM_OK) return s;
        return e == cudaSuccess ? BM_OK : BM_ECUDA;
    }
    const size_t smem = 2 * (size_t)N * 8;
    BM_CUDA_TRY(cudaFuncSetAttribute(k_poly_mul, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_poly_mul<<<count, N / 2 < 512 ? N / 2 : 512, smem, (cudaStream_t)stream>>>(key->d_view, d_a, d_b, d_out);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

extern "C" bm_status bm_mod_switch(const uint64_t *d_in, uint64_t *d_out, size_t words, uint64_t q_from,
                                   uint64_t q_to, void *stream) {
    if (q_from < 2 || q_to < 2 || (words && (!d_in || !d_out))) return BM_EINVAL;
    if (!words) return BM_OK;
    const size_t blocks = (words + 255) / 256 < 65535 ? (words + 255) / 256 : 65535;
    k_mod_switch<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_in, d_out, words, q_from, q_to);
    BM_CUDA_TRY(cudaGetLastError());
    return BM_OK;
}

// ---------------------------------------------------------------------------
// Arbitrary functions by two rounds (Section 4, last part)
// ---------------------------------------------------------------------------

namespace {
struct ArbLayout {
    size_t ws_bs, a, b, c, mp, F, total;
};

ArbLayout arb_layout(const bm_eval_key *key, uint32_t m, uint32_t t, uint32_t count) {
    ArbLayout L{};
    std::vector<bm_job> jobs(count);
    for (uint32_t i = 0; i < count; i++)
        jobs[i] = bm_job{0, m, 2 * t, 0, (uint64_t)i * (key->p.n + 1), 0, (uint64_t)i * (key->p.n + 1)};
    const bm_eval_key *keys[1] = {key};
    Plan pl;
    make_plan(keys, jobs.data(), count, pl);
    const size_t W = (size_t)count * (key->p.n + 1) * 8;
    L.ws_bs = align_up(pl.total, 256);
    L.a = L.ws_bs;
    L.b = L.a + align_up(W, 256);
    L.c = L.b + align_up(W, 256);
    L.mp = L.c + align_up(W, 256);
    L.F = L.mp + align_up((size_t)2 * t * 4, 256);
    L.total = L.F + align_up((size_t)count * 2 * t * 4, 256);
    return L;
}
}  // namespace

extern "C" size_t bm_arbitrary_workspace_bytes(const bm_eval_key *key, uint32_t m, uint32_t t, uint32_t count) {
    if (!key || !count || m < 1 || m > BM_MAX_M || 2ull * key->p.N * m > BM_MAX_QP || t < 2 || (t & 1)) return 0;
    return arb_layout(key, m, t, count).total;
}

extern "C" bm_status bm_bootstrap_arbitrary(const bm_eval_key *key, uint32_t m, uint32_t t, uint64_t q,
                                            const uint32_t *d_f, uint32_t count, const uint64_t *d_ct_in,
                                            uint64_t *d_ct_out, void *d_ws, size_t ws_bytes, void *stream) {
    if (!key || !d_f || !d_ct_in || !d_ct_out || !d_ws || ((uintptr_t)d_ws & 255)) return BM_EINVAL;
    if (!count) return BM_OK;
    const uint64_t qp = 2ull * key->p.N * m;
    if (m < 1 || m > BM_MAX_M || qp > BM_MAX_QP || t < 2 || (t & 1) || 2ull * t > qp || q < 2ull * t ||
        q >= key->p.Q)
        return BM_EINVAL;
    const ArbLayout L = arb_layout(key, m, t, count);
    if (ws_bytes < L.total) return BM_EWORKSPACE;
    DeviceGuard g(key->device);
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)d_ws;
    const u32 n = key->p.n, T = 2 * t;
    const size_t words = (size_t)count * (n + 1);
    u64 *A = (u64 *)(ws + L.a), *B = (u64 *)(ws + L.b), *Cb = (u64 *)(ws + L.c);
    u32 *mp = (u32 *)(ws + L.mp), *F = (u32 *)(ws + L.F);
    const unsigned blocks = (unsigned)((words + 255) / 256 < 4096 ? (words + 255) / 256 : 4096);
    k_two_round_tables<<<blocks, 256, 0, st>>>(d_f, t, count, mp, F);
    BM_CUDA_TRY(cudaGetLastError());
    std::vector<bm_job> jobs(count);
    for (uint32_t i = 0; i < count; i++)
        jobs[i] = bm_job{0, m, T, 0, (uint64_t)i * (n + 1), 0, (uint64_t)i * (n + 1)};
    const bm_eval_key *keys[1] = {key};
    bm_status s;
    // round 1: the top bit, mp over Z_{2t}
    if ((s = bm_mod_switch(d_ct_in, A, words, q, qp, stream)) != BM_OK) return s;
    if ((s = bm_bootstrap_batch(keys, 1, jobs.data(), count, A, mp, B, d_ws, L.ws_bs, stream)) != BM_OK) return s;
    if ((s = bm_mod_switch(B, B, words, key->p.Q, q, stream)) != BM_OK) return s;
    // y = x - (mp(x) + t/2): subtract the round-1 output and t/2 floor(q/2t)
    const u64 half = (u64)((unsigned __int128)(t / 2) * (q / T) % q);
    k_lwe_sub<<<blocks, 256, 0, st>>>(d_ct_in, B, Cb, count, n, q, half ? q - half : 0);
    BM_CUDA_TRY(cudaGetLastError());
    // round 2: f's negacyclic extension, one table per job
    if ((s = bm_mod_switch(Cb, A, words, q, qp, stream)) != BM_OK) return s;
    for (uint32_t i = 0; i < count; i++) jobs[i].lut_off = (uint64_t)i * T;
    if ((s = bm_bootstrap_batch(keys, 1, jobs.data(), count, A, F, B, d_ws, L.ws_bs, stream)) != BM_OK) return s;
    return bm_mod_switch(B, d_ct_out, words, key->p.Q, q, stream);
}

extern "C" bm_status bm_workspace_status(void *d_ws, void *stream) {
    if (!d_ws) return BM_EINVAL;
    u32 v = 0;
    BM_CUDA_TRY(cudaMemcpyAsync(&v, d_ws, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    BM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    BM_CUDA_TRY(cudaMemsetAsync(d_ws, 0, 4, (cudaStream_t)stream));
    BM_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return -(bm_status)v;
}

extern "C" bm_status bm_modmul_peak(int device, uint32_t iters, double *rate) {
    if (!rate || iters == 0) return BM_EINVAL;
    DeviceGuard g(device);
    int sms = 0;
    BM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const u32 blocks = (u32)sms * 8, threads = 256;
    u64 *d_out = nullptr;
    BM_CUDA_TRY(cudaMalloc(&d_out, (size_t)blocks * threads * 8));
    // the n = 630, N = 1024 key's modulus, Q = c 2^32 + 1
    const u64 Q = 18014359854776321ull, w = 123456789012345ull;
    const u64 wsh = (u64)(((unsigned __int128)w << 64) / Q);
    const u32 c = (u32)(Q >> 32);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_modmul_probe<<<blocks, threads>>>(d_out, iters / 8 + 1, c, w, wsh);   // warm-up
    cudaEventRecord(e0);
    k_modmul_probe<<<blocks, threads>>>(d_out, iters, c, w, wsh);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_out);
    if (err != cudaSuccess) return BM_ECUDA;
    *rate = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
    return BM_OK;
}

// ---------------------------------------------------------------------------
// Reusable batches: the plan is built and uploaded once; runs only launch.
// ---------------------------------------------------------------------------

extern "C" void bm_batch_free(bm_batch *b);

struct bm_batch {
    int device;
    uint32_t flags, n_persistent;
    Plan pl;
    Fork fork;
    Shapes shapes;     // the kernel shapes current when the batch was created
    KsShape ks;
    const uint64_t *d_ct_in;
    const uint32_t *d_lut;
    uint64_t *d_out;
    char *ws;
    cudaGraphExec_t exec;
    u32 max_cluster() const { return (flags & BM_BATCH_ONE_BLOCK) ? 1u : kMaxCluster; }
};

extern "C" bm_status bm_batch_create(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                     uint32_t count, const uint64_t *d_ct_in, const uint32_t *d_lut,
                                     uint64_t *d_ct_out, void *d_ws, size_t ws_bytes, uint32_t flags,
                                     bm_batch **out) {
    if (!out || (flags & ~(BM_BATCH_PERSISTENT | BM_BATCH_GRAPH | BM_BATCH_ONE_BLOCK))) return BM_EINVAL;
    int dev = 0;
    bm_status s = validate_jobs(keys, n_keys, jobs, count, &dev);
    if (s != BM_OK) return s;
    if (!count || !d_ct_in || !d_lut || !d_ct_out || !d_ws || ((uintptr_t)d_ws & 255)) return BM_EINVAL;
    bm_batch *b = new (std::nothrow) bm_batch();
    if (!b) return BM_ENOMEM;
    b->device = dev;
    b->flags = flags;
    make_plan(keys, jobs, count, b->pl, (flags & BM_BATCH_PERSISTENT) != 0);
    if (ws_bytes < b->pl.total) {
        delete b;
        return BM_EWORKSPACE;
    }
    b->n_persistent = (flags & BM_BATCH_PERSISTENT) ? persistent_prefix(b->pl) : 0;
    b->ks = ks_shape(keys, n_keys);
    b->shapes = Shapes::current();
    b->d_ct_in = d_ct_in;
    b->d_lut = d_lut;
    b->d_out = d_ct_out;
    b->ws = (char *)d_ws;
    b->exec = nullptr;
    DeviceGuard g(dev);
    cudaError_t e = cudaMemcpy(b->ws + b->pl.jobs_off, b->pl.dj.data(), sizeof(DevJob) * count,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->ws, 0, BM_WS_HEADER);
    // kernel attributes are set now, outside any later stream capture
    if (e == cudaSuccess && run_groups(b->pl, b->n_persistent, count, 0, nullptr, nullptr, b->ws, nullptr,
                                       true, b->max_cluster(), b->shapes) != BM_OK)
        e = cudaErrorUnknown;
    for (const ClassRange &cr : b->pl.classes) {
        if (e == cudaSuccess && bm_launch_persistent_class(cr.N, cr.variant, b->shapes.s[log2u(cr.N)], nullptr, 0, 0,
                                                           nullptr, nullptr, nullptr, nullptr, nullptr, dev, true,
                                                           nullptr) != BM_OK)
            e = cudaErrorUnknown;
    }
    if (b->pl.classes.size() > BM_MAX_CLASSES) e = cudaErrorInvalidValue;
    if (e == cudaSuccess && b->pl.classes.size() > 1) {
        const size_t nc = b->pl.classes.size();
        b->fork.side.resize(nc - 1, nullptr);
        b->fork.ev.resize(nc, nullptr);
        for (auto &sd : b->fork.side)
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sd, cudaStreamNonBlocking);
        for (auto &ev : b->fork.ev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        bm_batch_free(b);
        return BM_ECUDA;
    }
    *out = b;
    return BM_OK;
}

extern "C" bm_status bm_batch_run(bm_batch *b, void *stream) {
    if (!b) return BM_EINVAL;
    DeviceGuard g(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!(b->flags & BM_BATCH_GRAPH))
        return launch_all(b->pl, b->n_persistent, b->ks, b->device, 0xffffffffu, true, b->d_ct_in, b->d_lut,
                          b->d_out, b->ws, st, b->shapes, b->max_cluster(), &b->fork);
    if (!st) return BM_EINVAL;   // the legacy default stream cannot be captured
    if (!b->exec) {
        cudaGraph_t graph = nullptr;
        BM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        bm_status s = launch_all(b->pl, b->n_persistent, b->ks, b->device, 0xffffffffu, true, b->d_ct_in,
                                 b->d_lut, b->d_out, b->ws, st, b->shapes, b->max_cluster(), &b->fork);
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (s != BM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return BM_ECUDA;
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return BM_ECUDA;
        }
    }
    BM_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    return BM_OK;
}

extern "C" void bm_batch_free(bm_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaStream_t sd : b->fork.side)
        if (sd) cudaStreamDestroy(sd);
    for (cudaEvent_t ev : b->fork.ev)
        if (ev) cudaEventDestroy(ev);
    delete b;
}

// ---------------------------------------------------------------------------
// Kernel shapes
// ---------------------------------------------------------------------------

extern "C" bm_status bm_kernel_shape_info(uint32_t shape, uint32_t N, uint32_t *radix, uint32_t *threads,
                                          uint32_t *blocks_per_sm) {
    if (N < 256 || N > BM_MAX_N_BLOCK || (N & (N - 1)) || shape >= BM_NUM_SHAPES) return BM_EINVAL;
    if (shape != 0 && (N < 1024 || !br_shape_fits((int)log2u(N), (int)shape))) return BM_EINVAL;
    const BrShape b = br_shape((int)shape);
    if (radix) *radix = 1u << b.rb;
    if (threads) *threads = (uint32_t)b.threads;
    if (blocks_per_sm) *blocks_per_sm = (uint32_t)b.blocks;
    return BM_OK;
}

extern "C" bm_status bm_set_kernel_shape(uint32_t N, uint32_t shape) {
    if (N < 256 || N > BM_MAX_N_BLOCK || (N & (N - 1))) return BM_EINVAL;
    const u32 l = log2u(N);
    if (shape == BM_SHAPE_DEFAULT) shape = kDefaultShape[l];
    if (bm_kernel_shape_info(shape, N, nullptr, nullptr, nullptr) != BM_OK) return BM_EINVAL;
    g_shape[l].store(shape);
    return BM_OK;
}

extern "C" bm_status bm_get_kernel_shape(uint32_t N, uint32_t *shape) {
    if (N < 256 || N > BM_MAX_N_BLOCK || (N & (N - 1)) || !shape) return BM_EINVAL;
    *shape = g_shape[log2u(N)].load();
    return BM_OK;
}

// ---------------------------------------------------------------------------
// Bootstrapping without any device allocation.
//
// Some callers cannot allocate device memory when they want to bootstrap:
// code embedded in a host application whose memory pool already holds the
// GPU's memory, serving loops where a cudaMalloc or cudaFree would stall
// the whole device, and components that must keep their device footprint
// fixed after start-up.  For them, the job table, status word and
// accumulators of a batch live in one fixed array compiled into this
// library instead of a caller-supplied workspace.
// ---------------------------------------------------------------------------

static __device__ __align__(256) unsigned char g_noalloc_scratch[BM_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices];   // device address of the array, per device
void *g_noalloc_ctx[kMaxDevices];   // the context that address belongs to

// The current context, through the driver entry point of cuCtxGetCurrent
// (the runtime does not expose it).  Null when it cannot be queried.
void *current_context() {
    typedef int (*CtxGet)(void **);
    static CtxGet fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGet)f;
    });
    void *ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

__global__ void k_noalloc_status(const u32 *word, int32_t *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = -(int32_t)(*word);
}
}  // namespace

extern "C" bm_status bm_bootstrap_batch_noalloc(const bm_eval_key *const *keys, uint32_t n_keys,
                                                const bm_job *jobs, uint32_t count,
                                                const uint64_t *d_ct_in, const uint32_t *d_lut,
                                                uint64_t *d_ct_out, int32_t *d_status, void *stream) {
    int dev = 0;
    bm_status s = validate_jobs(keys, n_keys, jobs, count, &dev);
    if (s != BM_OK) return s;
    if (dev < 0 || dev >= kMaxDevices) return BM_EINVAL;
    Plan pl;
    make_plan(keys, jobs, count, pl);
    if (pl.total > BM_NOALLOC_SCRATCH_BYTES) {
        fprintf(stderr, "bootmmpm: batch needs %zu bytes of scratch, more than the %u built in\n",
                pl.total, (unsigned)BM_NOALLOC_SCRATCH_BYTES);
        return BM_EWORKSPACE;
    }
    DeviceGuard g(dev);
    void *scratch = nullptr;
    {
        // Host code sees only a stand-in for the array; its device address is
        // looked up once per device, with that device current, and again if
        // the device's context has changed since (a cudaDeviceReset destroys
        // the context the address belonged to).
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        void *ctx = current_context();
        if (!g_noalloc_ptr[dev] || ctx != g_noalloc_ctx[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                fprintf(stderr, "bootmmpm: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
                return BM_ECUDA;
            }
            g_noalloc_ptr[dev] = p;
            g_noalloc_ctx[dev] = ctx;
        }
        scratch = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    // The array keeps the previous call's contents: the status word must
    // start at zero (job table and accumulators are fully rewritten).
    BM_CUDA_TRY(cudaMemsetAsync(scratch, 0, BM_WS_HEADER, st));
    s = bootstrap_impl(keys, n_keys, jobs, count, 0xffffffffu, true, d_ct_in, d_lut, d_ct_out, scratch,
                       BM_NOALLOC_SCRATCH_BYTES, stream);
    if (s != BM_OK) return s;
    if (d_status) {
        k_noalloc_status<<<1, 32, 0, st>>>((const u32 *)scratch, d_status);
        BM_CUDA_TRY(cudaGetLastError());
    }
    return BM_OK;
}
