/*
 * bootmmpm.h -- C ABI of libbootmmpm.so: BootMMPM functional bootstrapping
 * (Liu and Li, "Large-Plaintext Functional Bootstrapping in FHE with Small
 * Bootstrapping Keys", arXiv 2310.12441) on NVIDIA GB300 (sm_103a).
 *
 * The library runs the data-parallel hot path of Algorithm 1 on the GPU:
 * test-vector construction and ACC initialisation, n CMux steps over the
 * monic monomial permutation matrices P(c) (blind rotation), sample
 * extraction and LWE key switching.  Key generation builds the evaluation
 * keys on the GPU from a seed (or from caller-supplied randomness);
 * encryption and decryption are client-side host routines.
 *
 * Conventions (Section 2 of the paper):
 *  - Z_Q values are uint64 in [0, Q); Q is prime, Q = 1 mod 2N, Q < 2^61.
 *  - An LWE ciphertext (a_1, ..., a_n, b) is n+1 consecutive uint64, b last;
 *    phase = b - <a, s>.  Inputs to bootstrapping live in Z_{q'}, q' = 2Nm
 *    (the output of Algorithm 1's first modulus switch); outputs in Z_Q.
 *  - An RLWE vector of m rows is [m][2][N] uint64: row r, component 0 = a,
 *    1 = b, coefficient of x^i at index i; phase_r = b_r - a_r z.
 *  - A look-up table is t uint32 entries f(0..t-1) in [0, t), negacyclic:
 *    f(k + t/2) = (t - f(k)) mod t  (Section 2, item (7)).
 *  - Secrets: s in {-1,0,1}^n (LWE, int8), z in {-1,0,1}^N (RLWE, int8).
 *
 * Ownership: key handles are created and freed by the library and own their
 * device memory.  Every other buffer belongs to the caller.  Device buffers
 * passed with a stream must stay valid until the stream's work completes.
 *
 * Errors: every call validates its arguments on the host and returns a
 * negative bm_status before launching anything.  Faults detected on the
 * device (a table that is not negacyclic, a bounded wait that expired) are
 * recorded in the status word at the start of the caller's workspace and
 * read back with bm_workspace_status(); no kernel traps.
 */
#ifndef BOOTMMPM_H
#define BOOTMMPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t bm_status;
#define BM_OK               0
#define BM_EINVAL          (-1)   /* an argument is out of range or inconsistent */
#define BM_ENOTPRIME       (-2)   /* Q is not prime or not 1 mod 2N */
#define BM_ENOMEM          (-3)   /* device allocation failed (key generation) */
#define BM_ENONNEGACYCLIC  (-4)   /* a look-up table is not negacyclic */
#define BM_ETIMEDOUT       (-5)   /* a bounded device wait expired */
#define BM_ECUDA           (-6)   /* a CUDA runtime call failed */
#define BM_EBUSY           (-7)   /* admission refused (serving loop) */
#define BM_EWORKSPACE      (-8)   /* the workspace is too small */

/* Evaluation-key parameters (Algorithm 1, REQUIRE block).  The keys do not
 * depend on m or t (Section 5, items (1)-(2)); one key set serves every job
 * shape (m, t) with the same N. */
typedef struct bm_key_params {
    uint32_t n;         /* LWE dimension */
    uint32_t N;         /* ring degree, power of two, 256..65536; above 8192 only jobs
                           with m = 1 (the single-polynomial layout) run, through
                           two-pass transforms in global memory */
    uint32_t log2_B;    /* blind-rotation gadget base B = 2^log2_B */
    uint32_t l_B;       /* gadget digits, B^l_B >= Q, 2 <= l_B <= 8 */
    uint32_t log2_Bks;  /* key-switching base B_ks = 2^log2_Bks, <= 8 */
    uint32_t l_ks;      /* key-switching digits of the approximate gadget, <= 16,
                           B_ks^l_ks < Q */
    uint64_t Q;         /* prime ring modulus */
} bm_key_params;

/* Randomness of key generation, all host arrays (C order):
 *   s        int8   [n]                     LWE secret, entries in {-1,0,1}
 *   z        int8   [N]                     RLWE secret, entries in {-1,0,1}
 *   bsk_mask uint64 [n][2][2 l_B][N]        uniform in [0, Q)
 *   bsk_err  int8   [n][2][2 l_B][N]        errors of the RGSW rows
 *   ksk_mask uint64 [N][l_ks][B_ks-1][n]    uniform in [0, Q)
 *   ksk_err  int8   [N][l_ks][B_ks-1]       errors of the LWE rows      */
typedef struct bm_key_randomness {
    const int8_t *s;
    const int8_t *z;
    const uint64_t *bsk_mask;
    const int8_t *bsk_err;
    const uint64_t *ksk_mask;
    const int8_t *ksk_err;
} bm_key_randomness;

typedef struct bm_secret_key bm_secret_key;
typedef struct bm_eval_key bm_eval_key;

/* One bootstrapping job (Definition 1): ciphertext, table, shape, key set. */
typedef struct bm_job {
    uint32_t key;       /* index into the key array of the call */
    uint32_t m;         /* polynomials in the test vector, 1..1024, with 2Nm <= 2^23
                           (1 for N above 8192) */
    uint32_t t;         /* plaintext modulus, even, 2 <= t <= 2Nm */
    uint32_t reserved;  /* must be 0 */
    uint64_t in_off;    /* element offset of the input LWE_{n,2Nm} (n+1 words) */
    uint64_t lut_off;   /* element offset of the table (t entries) */
    uint64_t out_off;   /* element offset of the output (n+1 words, or the
                           [m][2][N] ACC for bm_blind_rotate) */
} bm_job;

/* Key generation (Section 2 items (11) and (14); Algorithm 1 REQUIRE).
 * Builds on device `device`:
 *   BSK: for k in [n] and s_k+ = max(s_k,0), s_k- = max(-s_k,0), the RGSW
 *        encryptions under z: row j < l_B = (a + mu B^j, a z + e), row l_B+j =
 *        (a, a z + e + mu B^j); stored in the NTT domain scaled by N^-1;
 *   KSK: for i in [N], j in [l_ks], v in [1, B_ks), the LWE encryption under s
 *        of v z_i g_j, g_j = floor((Q B_ks^j + P/2) / P), P = B_ks^l_ks.
 * Copies the randomness, so the caller may free it on return.
 * Returns BM_EINVAL / BM_ENOTPRIME on bad parameters, BM_ENOMEM, BM_ECUDA. */
bm_status bm_keygen(const bm_key_params *params, const bm_key_randomness *rnd,
                    int device, bm_secret_key **sk_out, bm_eval_key **ek_out);
void bm_free_secret_key(bm_secret_key *sk);
void bm_free_eval_key(bm_eval_key *ek);

/* Keys drawn from a seed (Algorithm 1 REQUIRE block: s and z, and the masks
 * and errors of the keys of Section 2 items (11) and (14)).  The paper fixes
 * no generator; the library uses the counter-based Philox4x32-10 of Salmon,
 * Moraes, Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3",
 * SC'11), one 128-bit block per drawn value:
 *   block(kind, domain, i) = Philox4x32-10(counter = (i mod 2^32, i >> 32,
 *                            domain, kind), key = (seed mod 2^32, seed >> 32)).
 *   kind 1  s_k                 i = k                                 domain 0
 *   kind 2  z_i                 i = i                                 domain N
 *   kind 3  BSK mask word       i = ((k 2 + sgn) 2 l_B + row) N + c   domain N
 *   kind 4  BSK error           the same i                            domain N
 *   kind 5  KSK mask word       i = r n + c, r = (i_N l_ks + j)(B_ks - 1) + v - 1,  domain N
 *   kind 6  KSK error           i = r                                 domain N
 *   kind 7  encryption mask     i = ct n + c                          domain 0
 *   kind 8  encryption error    i = ct                                domain 0
 * Values from a block (w0, w1, w2, w3): uniform mod M is (w0 + w1 2^32 +
 * w2 2^64 + w3 2^96) mod M; ternary is floor(3 w0 / 2^32) - 1; binary is
 * floor(2 w0 / 2^32); an error is the discrete Gaussian exp(-k^2/(2 sigma^2))
 * on [-41, 41] by inversion, at r = w0 + w1 2^32, of the table
 * T_j = floor(2^64 F_j) (saturated at 2^64 - 1), F_j the mass of
 * [-41, -41 + j] summed in double from -41 upward.  sigma is the standard
 * deviation parameter, 0 < sigma <= BM_SIGMA_MAX (so the cut at 41 lies
 * beyond 10 sigma).  Two key sets with the same seed and n share s. */
#define BM_SECRET_BINARY 0u
#define BM_SECRET_TERNARY 1u
#define BM_SIGMA_MAX 4.0

/* Secret key only (host, no device): s (ternary, or binary with
 * BM_SECRET_BINARY) and z from `seed`.  BM_EINVAL / BM_ENOTPRIME on bad
 * parameters, BM_ENOMEM. */
bm_status bm_secret_key_seeded(const bm_key_params *params, uint32_t lwe_secret, uint64_t seed,
                               bm_secret_key **sk_out);

/* Secret key and evaluation key from `seed`: the secret as in
 * bm_secret_key_seeded, then the BSK and KSK built on `device` with every
 * mask and error drawn by the GPU threads that use them (no randomness
 * crosses the host-device link).  Same keys as bm_keygen given the arrays
 * these streams define.  Errors as bm_keygen. */
bm_status bm_keygen_seeded(const bm_key_params *params, uint32_t lwe_secret, double sigma, uint64_t seed,
                           int device, bm_secret_key **sk_out, bm_eval_key **ek_out);

/* Copies the secret key out: s (n int8, may be NULL) and z (N int8, may be
 * NULL). */
bm_status bm_secret_key_get(const bm_secret_key *sk, int8_t *s_out, int8_t *z_out);

/* Device bytes held by an evaluation key (BSK + KSK + tables). */
size_t bm_eval_key_bytes(const bm_eval_key *ek);

/* LWE_{n,q} encryption on the host (Section 2, item (8)):
 * ct_i = (a_i, <a_i, s> + msg_i floor(q/t) + e_i) mod q, for `count` messages.
 * mask: uint64 [count][n] in [0, q); err: int8 [count]; ct_out: [count][n+1]. */
bm_status bm_encrypt(const bm_secret_key *sk, uint64_t q, uint32_t t,
                     const uint32_t *msg, const uint64_t *mask, const int8_t *err,
                     size_t count, uint64_t *ct_out);

/* bm_encrypt with the masks and errors drawn from `seed` (kinds 7 and 8 of
 * the stream layout above; errors of parameter sigma). */
bm_status bm_encrypt_seeded(const bm_secret_key *sk, uint64_t q, uint32_t t, const uint32_t *msg,
                            size_t count, double sigma, uint64_t seed, uint64_t *ct_out);

/* LWE decryption on the host: msg = floor((phase t + floor(q/2)) / q) mod t.
 * ct: [count][n+1] in [0, q). */
bm_status bm_decrypt(const bm_secret_key *sk, uint64_t q, uint32_t t,
                     const uint64_t *ct, size_t count, uint32_t *msg_out);

/* Bytes of device workspace that bm_bootstrap_batch / bm_blind_rotate need
 * for these jobs (status word, job table, per-job accumulators). */
size_t bm_workspace_bytes(const bm_eval_key *const *keys, uint32_t n_keys,
                          const bm_job *jobs, uint32_t count);

/* Algorithm 1 for `count` jobs in one launch sequence on `stream`
 * (a cudaStream_t, or NULL for the default stream):
 *   ACC <- P(b) (0, v_test floor(Q/t))            (test vector Eq. (equ:test-use))
 *   for k = 1..n: ACC <- CMux(ct_k+, ct_k-; P(-a_k), I, P(a_k)) ACC   (Eq. (cmux:BP))
 *   ct  <- SampleExtract(row 0 of ACC)            (Eq. (equ-sam-extr))
 *   ct  <- KeySwitch_{z -> s}(ct)                 (Eq. (equ-key-swi))
 * The input modulus switch is the identity (inputs are given in Z_{2Nm});
 * the final switch Q -> q is not applied: outputs are LWE_{n,Q} under s.
 * d_ct_in (uint64), d_lut (uint32), d_ct_out (uint64): device arrays indexed
 * by the jobs' offsets.  d_ws: device workspace of ws_bytes bytes, 256-byte
 * aligned.  Asynchronous; host-side validation errors return before any
 * launch, device-side ones land in the workspace status word. */
bm_status bm_bootstrap_batch(const bm_eval_key *const *keys, uint32_t n_keys,
                             const bm_job *jobs, uint32_t count,
                             const uint64_t *d_ct_in, const uint32_t *d_lut,
                             uint64_t *d_ct_out, void *d_ws, size_t ws_bytes,
                             void *stream);

/* Algorithm 1 with other transitive generators (Theorem 1; Lemma 3;
 * Example 2, Eq. (equ:test-gene)).  A generator is given by m exponents
 * u_0..u_{m-1} in [0, 2N): P(1) = (x^{u_i} delta_{i-1 mod m, j}), i.e. row 0
 * holds x^{u_0} in column m-1 and row i >= 1 holds x^{u_i} in column i-1.
 * By Theorem 1 it acts transitively on the monic monomial indicator vectors
 * (so that the test vector has the look-up property) iff sum u is odd;
 * other generators are refused (BM_EINVAL).  Then P(c) = P(1)^c has row i
 * equal to x^{E_c(i)} e_{(i-c) mod m}, E_c(i) = sum_{t in [c]} u_{(i-t) mod m}
 * (Lemma 3), and the test vector is v_0 = sum_{a in [N], b in [m]}
 * f'(-(a m + b)) x^{a S + E_b(b)} e_b with S = sum u.
 * gens: host array of exponents; job i uses gens[gen_off[i] .. + m_i), or
 * Example 1's generator u = (1, 0, ..., 0) when gen_off[i] ==
 * BM_GEN_EXAMPLE1 (bm_bootstrap_batch uses it for every job).  Otherwise as
 * bm_bootstrap_batch, with a workspace of bm_workspace_bytes_gen(...) bytes. */
#define BM_GEN_EXAMPLE1 (~(uint64_t)0)
size_t bm_workspace_bytes_gen(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                              uint32_t count, const uint32_t *gens, const uint64_t *gen_off);
bm_status bm_bootstrap_batch_gen(const bm_eval_key *const *keys, uint32_t n_keys, const bm_job *jobs,
                                 uint32_t count, const uint32_t *gens, const uint64_t *gen_off,
                                 const uint64_t *d_ct_in, const uint32_t *d_lut, uint64_t *d_ct_out,
                                 void *d_ws, size_t ws_bytes, void *stream);

/* Same computation with host buffers: copies the inputs (h_ct_in, h_lut) to
 * the workspace, bootstraps, copies the outputs back to h_ct_out, and
 * synchronises the stream.  The workspace must hold
 * bm_workspace_bytes(...) + bm_host_staging_bytes(...). */
size_t bm_host_staging_bytes(const bm_eval_key *const *keys, uint32_t n_keys,
                             const bm_job *jobs, uint32_t count);
bm_status bm_bootstrap_batch_host(const bm_eval_key *const *keys, uint32_t n_keys,
                                  const bm_job *jobs, uint32_t count,
                                  const uint64_t *h_ct_in, size_t ct_in_words,
                                  const uint32_t *h_lut, size_t lut_words,
                                  uint64_t *h_ct_out, size_t ct_out_words,
                                  void *d_ws, size_t ws_bytes, void *stream);

/* Blind rotation only (Algorithm 1, phase accumulation): writes each job's
 * final ACC, [m][2][N] uint64, at d_acc_out + job.out_off.  `steps` limits
 * the CMux loop to its first `steps` iterations (steps >= n runs all). */
bm_status bm_blind_rotate(const bm_eval_key *const *keys, uint32_t n_keys,
                          const bm_job *jobs, uint32_t count, uint32_t steps,
                          const uint64_t *d_ct_in, const uint32_t *d_lut,
                          uint64_t *d_acc_out, void *d_ws, size_t ws_bytes,
                          void *stream);

/* Sample extraction (Section 2 item (13), Eq. (equ-sam-extr)): for each of
 * `count` RLWE ciphertexts (a, b) at d_rlwe + i*2N, writes the LWE_{N,Q}
 * sample (a_0, -a_{N-1}, ..., -a_1, b_0) at d_lwe_out + i*(N+1). */
bm_status bm_sample_extract(const bm_eval_key *key, const uint64_t *d_rlwe,
                            uint32_t count, uint64_t *d_lwe_out, void *stream);

/* LWE key switching z -> s (Section 2 item (11), Eq. (equ-key-swi)) with the
 * approximate gadget: a~_i = floor((a_i P + floor(Q/2)) / Q) mod P split into
 * l_ks base-B_ks digits d_ij; out = (0^n, b) - sum_ij KSK(i, j, d_ij).
 * d_lwe_in: [count][N+1]; d_out: [count][n+1]. */
bm_status bm_key_switch(const bm_eval_key *key, const uint64_t *d_lwe_in,
                        uint32_t count, uint64_t *d_out, void *stream);

/* Negacyclic products in R_{N,Q} (Section 2 item (6)) through the library's
 * NTT: d_out[i] = d_a[i] * d_b[i] for `count` pairs of N coefficients.  For
 * N above 8192 the call allocates count N words of device scratch and
 * returns after the stream has finished. */
bm_status bm_poly_mul(const bm_eval_key *key, const uint64_t *d_a,
                      const uint64_t *d_b, uint32_t count, uint64_t *d_out,
                      void *stream);

/* Reusable batch (native executor around Algorithm 1): the job table is
 * built, ordered and uploaded to the workspace once; every bm_batch_run then
 * only launches kernels on the bound buffers.  Flags:
 *   BM_BATCH_PERSISTENT  one persistent blind-rotation launch for all jobs of
 *                        ring degree 1024..4096 (one 512-thread block per SM
 *                        pulls jobs from a counter, longest first), so uneven
 *                        mixes of key sets and shapes run as one launch;
 *   BM_BATCH_GRAPH       the first run records the launches in a CUDA graph
 *                        on `stream` (which must not be the legacy default
 *                        stream) and later runs replay it;
 *   BM_BATCH_ONE_BLOCK   every job runs on one block.  Without it (and in
 *                        bm_bootstrap_batch), a launch of fewer jobs than the
 *                        GPU holds gives each job a thread-block cluster of
 *                        up to 8 blocks that split its m rows (the rows of one
 *                        CMux step are independent, Eq. (ex1:BPc)), which cuts
 *                        the latency of small batches; results are identical.
 * The buffers and the workspace stay bound to the batch until bm_batch_free;
 * runs of one batch must not overlap on the GPU (they share the workspace). */
typedef struct bm_batch bm_batch;
#define BM_BATCH_PERSISTENT 1u
#define BM_BATCH_GRAPH 2u
#define BM_BATCH_ONE_BLOCK 4u
bm_status bm_batch_create(const bm_eval_key *const *keys, uint32_t n_keys,
                          const bm_job *jobs, uint32_t count,
                          const uint64_t *d_ct_in, const uint32_t *d_lut,
                          uint64_t *d_ct_out, void *d_ws, size_t ws_bytes,
                          uint32_t flags, bm_batch **out);
bm_status bm_batch_run(bm_batch *batch, void *stream);
void bm_batch_free(bm_batch *batch);

/* Modulus switch (Section 2 item (9)) of `words` consecutive words, on the
 * device of the current context: out = floor((x q_to + floor(q_from/2)) /
 * q_from) mod q_to, x in [0, q_from) (larger words are first reduced).  Used
 * before bootstrapping (q -> 2Nm, Algorithm 1's first line) and after it
 * (Q -> q, Algorithm 1's last line); in place is allowed. */
bm_status bm_mod_switch(const uint64_t *d_in, uint64_t *d_out, size_t words,
                        uint64_t q_from, uint64_t q_to, void *stream);

/* Any function f: Z_t -> Z_t, negacyclic or not, by the two-round method of
 * Section 4 (last part; Eqs. (rel:mp), (rel:sign)).  Each input is an
 * LWE_{n,q} encryption of m in [0, t) under plaintext modulus 2t (its top bit
 * may be unknown: any x in Z_{2t} is read as m = x mod t).  Round 1
 * bootstraps mp (-t/2 on [-t/2, t/2), t/2 elsewhere) to extract the top bit,
 * using sign(x) t = mp(x) + t/2; that is switched back to q and subtracted,
 * leaving y in [-t/2, t/2) with y = m mod t; round 2 bootstraps the
 * negacyclic extension F of f from [-t/2, t/2).  Each bootstrap switches
 * q -> 2Nm first and Q -> q after (Algorithm 1's modulus switches).
 * Outputs: LWE_{n,q} encryptions of f(m) under plaintext modulus 2t.
 * d_f: count tables of t uint32 entries in [0, t); d_ct_in / d_ct_out:
 * [count][n+1] words mod q; needs 2t <= 2Nm, 2t <= q < Q, and a workspace of
 * bm_arbitrary_workspace_bytes(key, m, t, count) bytes. */
size_t bm_arbitrary_workspace_bytes(const bm_eval_key *key, uint32_t m, uint32_t t,
                                    uint32_t count);
bm_status bm_bootstrap_arbitrary(const bm_eval_key *key, uint32_t m, uint32_t t,
                                 uint64_t q, const uint32_t *d_f, uint32_t count,
                                 const uint64_t *d_ct_in, uint64_t *d_ct_out,
                                 void *d_ws, size_t ws_bytes, void *stream);

/* Kernel shapes of the blind rotation (the autotuner's candidates; the paper
 * has no counterpart: they change how the GPU runs Algorithm 1, never a
 * result bit).  Shape s runs each job on blocks of `threads` threads holding
 * `radix` coefficients of a polynomial each in the transforms, with
 * `blocks_per_sm` blocks resident per SM:
 *   0: radix 16, 512 threads, 1 block/SM     (every ring degree)
 *   1: radix 8, 1024 threads, 1 block/SM     (N = 1024..8192)
 *   2: radix 16, 256 threads, 2 blocks/SM    (N = 1024)
 *   3: radix 8, 512 threads, 2 blocks/SM     (N = 1024)
 *   4: radix 8, 512 threads, 1 block/SM      (N = 1024..4096)
 * Shapes 1..4 are compiled for keys whose Q = c 2^32 + 1; other keys run
 * shape 0.  bm_kernel_shape_info describes shape s at ring degree N
 * (BM_EINVAL when it does not fit).  bm_set_kernel_shape selects the shape
 * that later launches at ring degree N use (BM_SHAPE_DEFAULT: the built-in
 * choice, shape 1 for N = 1024..8192 and 0 below); reusable batches keep the shapes current at bm_batch_create.
 * The setting is process-wide. */
#define BM_NUM_SHAPES 5
#define BM_SHAPE_DEFAULT 0xffffffffu
bm_status bm_kernel_shape_info(uint32_t shape, uint32_t N, uint32_t *radix, uint32_t *threads,
                               uint32_t *blocks_per_sm);
bm_status bm_set_kernel_shape(uint32_t N, uint32_t shape);
bm_status bm_get_kernel_shape(uint32_t N, uint32_t *shape);

/* Reads (synchronising `stream`) and clears the device status word of a
 * workspace: BM_OK or the first device-side error recorded. */
bm_status bm_workspace_status(void *d_ws, void *stream);

/* Throughput probe of the modular multiplication the blind rotation uses
 * (three-product Shoup for Q = c 2^32 + 1, the integer-ALU roofline
 * denominator): runs `iters` steps of eight independent chains on every
 * thread of a full-device grid and returns modmuls/s in *rate. */
bm_status bm_modmul_peak(int device, uint32_t iters, double *rate);

/* Bootstrapping for callers that cannot allocate device memory (no
 * counterpart in the paper; a property of this library's interface).
 * Such callers include code running inside a host application whose memory
 * pool already owns the GPU's memory, serving loops in which a cudaMalloc or
 * cudaFree would stall every stream on the device, and components whose
 * device footprint must stay fixed after start-up.
 *
 * Same computation and arguments as bm_bootstrap_batch, but the job table,
 * status word and accumulators live in a fixed array of
 * BM_NOALLOC_SCRATCH_BYTES bytes inside the library (every GPU that loads
 * the library holds it until the process exits).  The call performs no
 * device allocation of any kind.  A batch needing more than the array
 * (bm_workspace_bytes(...) > BM_NOALLOC_SCRATCH_BYTES) is rejected with
 * BM_EWORKSPACE before anything is launched.
 *  - The first call on a device looks up the array's device address with
 *    that device current; make that first call before any stream capture.
 *    The lookup is repeated when the device's context has changed since
 *    (after a cudaDeviceReset), so that call too belongs outside a capture.
 *  - Every call shares the one array: calls whose work overlaps on the GPU
 *    (concurrent streams, or threads) race and corrupt each other.  Order
 *    them on one stream or synchronise between them.
 *  - d_status (device int32, may be NULL) receives BM_OK or the first
 *    device-side error of this call, written after the batch on `stream`. */
#define BM_NOALLOC_SCRATCH_BYTES (16u << 20)
bm_status bm_bootstrap_batch_noalloc(const bm_eval_key *const *keys, uint32_t n_keys,
                                     const bm_job *jobs, uint32_t count,
                                     const uint64_t *d_ct_in, const uint32_t *d_lut,
                                     uint64_t *d_ct_out, int32_t *d_status, void *stream);

const char *bm_status_str(bm_status s);

#ifdef __cplusplus
}
#endif
#endif /* BOOTMMPM_H */
