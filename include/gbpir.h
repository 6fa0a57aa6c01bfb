/*
 * gbpir.h -- C ABI of the GB300 (sm_103a) RLWE-PIR first-dimension scan.
 *
 * The server's online linear scan of single-server PIR in its poly-HE
 * (RLWE) form, as described in VIPIR (arXiv 2606.11536):
 *   - the database is NTT-encoded once ("DB bloating", Sec. 3.3; fused RNS lift
 *     and NTT, Sec. 4.3);
 *   - a query is D1 RLWE ciphertexts, one per first-dimension index (a one-hot
 *     encryption, Sec. 2.5 / Sec. 3.2 "poly-HE folding");
 *   - the answer folds the first dimension: for every column c,
 *     out_c = sum_i DB[i][c] * ct_i in R_q^2 (plaintext-ciphertext products,
 *     App. A.2), computed per RNS prime q_j and NTT slot k as
 *     out[b][c][k] = sum_i DB[i][c][k] * Q[b][i][k] mod q_j
 *     ("(#RNS*N)-parallel INT32 modular GEMMs", Sec. 4 and Sec. 4.2),
 *     then inverse-NTT'd back to coefficient form.
 *
 * Conventions shared by every call:
 *   - A polynomial ring is Z_q[X]/(X^n + 1), n a power of two in [2^11, 2^13];
 *     q = q_0 * ... * q_{L-1} with 30-bit primes q_j = 1 mod 2n and q_j = 1 mod p
 *     (App. A.4).  Residues are uint32 values, canonical in [0, q_j).
 *   - An RNS polynomial is laid out [L][n] (row j holds the residues mod q_j).
 *   - NTT order: NTT(a)[k] = sum_t a_t * psi_j^((2*brv(k) + 1) * t) mod q_j, with
 *     brv the log2(n)-bit reversal and psi_j a primitive 2n-th root of unity.
 *   - A ciphertext is [2][L][n]: component 0 = a(X), component 1 = b(X), with
 *     a*s + b = Delta*m + e (mod q), Delta = floor(q/p) (App. A.2).
 *   - Calls on device buffers are asynchronous and ordered on `stream` (a
 *     cudaStream_t, NULL = the legacy default stream).  Calls on host buffers are
 *     synchronous: they return once the host output is written.
 *   - Every call returns a status; nothing aborts, traps or exits.
 *   - All device pointers must be 16-byte aligned.
 */
#ifndef GBPIR_H
#define GBPIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIR_MAX_L 4

typedef enum {
  PIR_OK = 0,
  PIR_ERR_ARG = 1,         /* bad pointer, size, shape or parameter              */
  PIR_ERR_OOM = 2,         /* a device or host allocation failed                 */
  PIR_ERR_ADMISSION = 3,   /* the DB does not fit the device memory left         */
  PIR_ERR_CUDA = 4,        /* a CUDA runtime call failed (see pir_last_cuda_error) */
  PIR_ERR_TIMEOUT = 5,     /* a bounded wait ran out                             */
  PIR_ERR_HANDLE = 6,      /* unknown or already freed DB handle                 */
  PIR_ERR_UNSUPPORTED = 7  /* valid request this build does not implement        */
} pir_status_t;

/* Parameters of one PIR instance.  n = ring degree, L = number of RNS primes,
 * log2p = log2 of the plaintext modulus p, D1 x D2 = database shape in plaintext
 * polynomials (D1 = first dimension, folded by the scan; D2 = columns).  q[j] and
 * psi[j] for j < L; unused entries are zero. */
typedef struct {
  uint32_t n, L, log2p, D1, D2;
  uint32_t q[PIR_MAX_L];
  uint32_t psi[PIR_MAX_L];
} pir_params_t;

/* Resident-DB layouts, chosen once at setup (the GEMM path follows the layout). */
typedef enum {
  PIR_LAYOUT_PLAIN = 0,  /* u32 residues [L*n slots][D1][D2]: CUDA-core u32 x u32 -> u64 path */
  PIR_LAYOUT_LIMB = 1,   /* u8 limb planes [L*n slots][4][D2][D1]: INT8 tensor-pipe path    */
  PIR_LAYOUT_TENSOR = 2  /* signed base-256 digits in bf16, 8 bytes per residue, laid out as
                            tensor-core operand tiles: the tcgen05 bf16 path (needs
                            D1 % 64 == 0 and D2 % 32 == 0)                                     */
} pir_layout_t;

typedef struct pir_db *pir_db_t;

/* Fill *out for ring degree n, plaintext modulus 2^log2p, shape D1 x D2 and L
 * primes: q_j are the L largest primes in (2^29, 2^30) with q_j = 1 mod max(2n, p),
 * in decreasing order; psi_j = h^((q_j - 1)/(2n)) for the smallest h >= 2 with
 * psi_j^n = -1 (App. A.4; the root choice is this library's reading, the paper
 * does not fix one).  Errors: PIR_ERR_ARG for n not in {2^11, 2^12, 2^13},
 * L not in [1, 4], log2p not in [1, 28] or 2n not dividing a power of two >= p,
 * or D1/D2 zero; PIR_ERR_UNSUPPORTED if fewer than L such primes exist. */
pir_status_t pir_make_params(uint32_t n, uint32_t log2p, uint32_t D1, uint32_t D2, uint32_t L,
                             pir_params_t *out);

/* Load and NTT-encode a database (Sec. 3.3; RNS lift fused with the NTT, Sec. 4.3).
 *   raw_db:     D1*D2*n*log2p/8 bytes, a little-endian bit stream of log2p-bit
 *               coefficients, polynomial after polynomial, polynomial (i, c) at
 *               position i*D2 + c.  Host or device memory (raw_on_device).
 *   layout:     PIR_LAYOUT_PLAIN, PIR_LAYOUT_LIMB or PIR_LAYOUT_TENSOR.  The tensor
 *               layout holds twice the bytes of the others and runs the batched
 *               answer on the bf16 tensor cores (K-chunks of at most 1024 rows keep
 *               the f32 sums of digit products exact).
 *   stream:     cudaStream_t for the encode kernels; the call returns after the
 *               DB is resident (it synchronizes the stream).
 *   out_handle: receives the handle; the library owns the resident DB until
 *               pir_free_db.  The caller keeps ownership of raw_db.
 * Errors: PIR_ERR_ARG (NULL pointers, raw_bytes mismatch, invalid params),
 * PIR_ERR_UNSUPPORTED (D2 not a multiple of 4: the kernels move columns four at a
 * time; the limb layout with D1 not a multiple of 32: its tensor steps take 32 rows;
 * the tensor layout with D1 not a multiple of 64 or D2 not a multiple of 32),
 * PIR_ERR_ADMISSION (resident bytes exceed the free device memory less a reserve,
 * counted after the scratch the library keeps cached for answers and graphs has been
 * given back), PIR_ERR_OOM, PIR_ERR_CUDA. */
pir_status_t pir_setup_db(const pir_params_t *params, const void *raw_db, size_t raw_bytes, int raw_on_device,
                          int layout, void *stream, pir_db_t *out_handle);

/* Answer a batch of B queries against a resident DB (the online scan).
 *   queries:   [B][D1][2][L][n] uint32, coefficient form, canonical residues.
 *   responses: [B][D2][2][L][n] uint32, coefficient form, canonical; written.
 *   on_device: 1 = both buffers are device memory (asynchronous on stream);
 *              0 = both are host memory (copied in and out; synchronous; pinned
 *              host memory gives the fastest copies).
 * Computes, for every b, c: responses[b][c] = sum_i DB[i][c] * queries[b][i] in
 * R_q^2 (Sec. 3.2; Sec. 4 "INT32 modular GEMM"), through forward NTT of the
 * queries, the per-slot modular GEMM on the layout's GEMM path, reduction to
 * [0, q_j) and inverse NTT.  Scratch device memory is drawn from the stream-ordered
 * allocator and returned before the call's work completes.
 * Errors: PIR_ERR_HANDLE, PIR_ERR_ARG (B = 0, NULL or misaligned buffers),
 * PIR_ERR_OOM, PIR_ERR_CUDA. */
pir_status_t pir_answer(pir_db_t db, const uint32_t *queries, uint32_t B, uint32_t *responses, int on_device,
                        void *stream);

/* Options for pir_answer_ex.  Zero-initialised = the defaults of pir_answer. */
typedef struct {
  uint32_t k_chunk;  /* 0 = automatic: whole D1 when its scratch fits half of the
                        available device memory, else equal chunks that do, of at
                        least 512 ciphertexts (or D1); else fold D1 in chunks of
                        this many ciphertexts (bounds the scratch to one chunk)     */
  uint32_t tile;     /* 0 = built-in choice; else a GEMM tile id (pir_gemm_tiles) that
                        holds the batch: plain 1, 2, 3 and 7 take at most 2, 4, 8 and
                        8 query rows (2B), 7 also D2 <= 512; limb 2 and 3 need the
                        rows padded to 16 to be multiples of 32 and 64; tensor 1 is
                        the 1-SM GEMM, 2 the CTA-pair (2-SM) GEMM, which needs
                        D2 % 64 == 0, 3 and 4 the 1-SM GEMM in clusters of 2 and 4
                        CTAs that multicast the query digits, which need D2 % 64
                        and D2 % 128 == 0, 5 the CTA-pair GEMM loading by tensor
                        maps, which needs D2 % 64 == 0 and the query rows padded to
                        8 (Mp) with 4 Mp <= 256 or a multiple of 256; otherwise
                        PIR_ERR_ARG */
  uint32_t flags;    /* PIR_ANSWER_STAGE_TIMES: record CUDA events around each stage on
                        `stream`, read with pir_stage_times; PIR_ANSWER_TEST_STALL,
                        PIR_ANSWER_MODSWITCH, PIR_ANSWER_CHECK_INPUTS: see below.
                        Other bits must be 0. */
} pir_answer_opts_t;

#define PIR_ANSWER_STAGE_TIMES 1u
/* Test hook for the bounded-wait error path: the TMA-staged scan's consumers wait
 * on a barrier nothing arrives on, time out after about a second, set the device
 * error word and return (the answer is then invalid; pir_check_device reports
 * PIR_ERR_TIMEOUT).  Needs a shape the TMA scan holds (2B <= 8, D2 <= 512). */
#define PIR_ANSWER_TEST_STALL 2u
/* Modulus switching of the responses to the single prime q_0, fused into the
 * inverse NTT (Sec. 4.3; App. D.5, error analysis of RLWE modulus switching): the
 * responses are then [B][D2][2][n] uint32 over q_0, coefficient form, canonical
 * (half the bytes at L = 2), as ntt_inv_modswitch below computes them. */
#define PIR_ANSWER_MODSWITCH 4u
/* Input validation: before computing, check on the device that every query
 * residue is canonical (below its prime q_j; the answer is only defined for such
 * inputs) and return PIR_ERR_ARG if one is not.  Costs one extra read of the
 * queries and a stream synchronization, so it is off by default.  Accepted by
 * pir_answer_ex on device buffers and on host batches up to 4 GiB (checked after
 * the upload); refused (PIR_ERR_ARG) by the streamed answer, graphs and the
 * no-allocation entry point. */
#define PIR_ANSWER_CHECK_INPUTS 8u

/* Stages of one answer, in order: forward NTT of the queries, query transpose to
 * the slot-major layout, modular GEMM (with its reduction epilogue), result
 * transpose, inverse NTT. */
#define PIR_STAGES 5

/* pir_answer with options.  With host buffers and k_chunk = 0:
 *   - batches of 16 and more (8 MiB to 4 GiB of queries) run as sub-batches of at
 *     least 8 queries, whose upload, answer and download overlap on three streams;
 *   - smaller batches of 8 MiB to 4 GiB upload in four pieces on a copy stream,
 *     each piece's forward NTT waiting only for its own copy;
 *   - host batches above 4 GiB run as a streamed answer (pir_answer_begin below) in
 *     pieces of at most 1 GiB (the tensor layout: up to 1024 ciphertexts, as the
 *     free memory allows), so the device holds one piece at a time; the first two
 *     pieces are 1/16 and 1/4 of that, so the scan starts after a short upload. */
pir_status_t pir_answer_ex(pir_db_t db, const uint32_t *queries, uint32_t B, uint32_t *responses, int on_device,
                           void *stream, const pir_answer_opts_t *opts);

/* Streamed answer: the queries arrive in pieces along D1 (Sec. 4.4, stream-wise
 * buffering of the first-dimension scan), so a batch whose query ciphertexts do
 * not fit device memory, or whose upload should overlap the scan, needs only one
 * piece resident at a time.
 *   pir_answer_begin: opens a session for B queries against db; kc_max bounds the
 *     ciphertexts per piece (the device scratch is sized by it).  opts as for
 *     pir_answer_ex except that k_chunk must be 0 and PIR_ANSWER_TEST_STALL is
 *     refused.  Work runs on `stream`.
 *   pir_answer_chunk: ciphertexts i0 .. i0+kc-1 of every query, [B][kc][2][L][n]
 *     uint32 coefficient form, canonical.  Pieces come in order: i0 is the first
 *     ciphertext not yet given, 1 <= kc <= kc_max, i0 + kc <= D1; on the limb
 *     layout kc is a multiple of 32.  Device buffers (on_device = 1) are read in
 *     `stream`'s order and must stay valid until the work is done.  Host buffers
 *     are copied on a copy stream through two staging buffers, so the copy of
 *     one piece overlaps the scan of the previous one; the call returns once its
 *     copy is complete and the buffer may be reused.
 *   pir_answer_end: after all D1 ciphertexts, writes the responses as pir_answer_ex
 *     does ([B][D2][2][L][n], or [B][D2][2][n] over q_0 with PIR_ANSWER_MODSWITCH);
 *     host buffers are filled when it returns.  Releases the session in every
 *     case.  pir_answer_abort releases it without a result.
 * The result equals pir_answer_ex on the whole query buffer.  The DB must outlive
 * the session.  A failed pir_answer_chunk leaves the session failed: pir_answer_end
 * then returns that status.
 * Errors: PIR_ERR_HANDLE (session or DB), PIR_ERR_ARG (B = 0, kc_max = 0, NULL or
 * misaligned buffers, pieces out of order or out of range, end before D1
 * ciphertexts), PIR_ERR_OOM, PIR_ERR_CUDA. */
typedef struct pir_session *pir_session_t;
pir_status_t pir_answer_begin(pir_db_t db, uint32_t B, uint32_t kc_max, void *stream, const pir_answer_opts_t *opts,
                              pir_session_t *out);
pir_status_t pir_answer_chunk(pir_session_t session, const uint32_t *queries, uint32_t i0, uint32_t kc,
                              int on_device);
pir_status_t pir_answer_end(pir_session_t session, uint32_t *responses, int on_device);
pir_status_t pir_answer_abort(pir_session_t session);

/* A whole answer captured once into a CUDA graph (all its kernels, scratch
 * allocation and release as graph nodes) and replayed with one launch: the
 * batched, graph-captured launch the scan is served with.  The graph is bound to
 * the device buffers given here (queries [B][D1][2][L][n], responses
 * [B][D2][2][L][n], or [B][D2][2][n] with PIR_ANSWER_MODSWITCH); every
 * pir_graph_launch answers whatever the query buffer holds at that point in
 * `stream`'s order.  opts as for pir_answer_ex, except that
 * PIR_ANSWER_STAGE_TIMES and PIR_ANSWER_TEST_STALL are refused (PIR_ERR_ARG).
 * The caller keeps ownership of the buffers and must keep them (and the DB) alive
 * until pir_graph_destroy, which also returns the graph's own scratch memory to the
 * device.  Errors: PIR_ERR_HANDLE, PIR_ERR_ARG, PIR_ERR_CUDA. */
typedef struct pir_graph *pir_graph_t;
pir_status_t pir_graph_create(pir_db_t db, const uint32_t *queries, uint32_t B, uint32_t *responses,
                              const pir_answer_opts_t *opts, pir_graph_t *out);
pir_status_t pir_graph_launch(pir_graph_t graph, void *stream);
pir_status_t pir_graph_destroy(pir_graph_t graph);

/* Autotuner: times every GEMM tile valid for this DB's layout and batch size B,
 * and K-chunk choices (whole D1, halves, quarters), `reps` answers each on scratch
 * buffers (all-zero queries; the scan's cost does not depend on the data), with
 * CUDA events on `stream`.  Candidates go in order (tiles by id, then whole D1
 * before halves and quarters) and a later one wins only if at least 1% faster, so
 * timing noise does not flip the choice between equals.  Writes the winner
 * (tile, k_chunk) to *best and caches it in the handle, so later calls for the
 * same B return at once.  Synchronous.
 * Errors: PIR_ERR_HANDLE, PIR_ERR_ARG (B = 0, best NULL), PIR_ERR_OOM, PIR_ERR_CUDA. */
pir_status_t pir_autotune(pir_db_t db, uint32_t B, void *stream, uint32_t reps, pir_answer_opts_t *best);

/* pir_answer_noalloc -- the answer without any device allocation.  The paper has
 * no counterpart; this entry point exists for callers that cannot allocate device
 * memory while serving: processes that reserve their whole device-memory budget up
 * front (a server handing all free HBM to resident databases, a host application
 * whose allocator owns the device) and latency-critical paths that cannot afford
 * an allocator call.  Same inputs, outputs and result as pir_answer with device
 * buffers (on_device = 1), asynchronous on `stream`.
 *   Scratch: one static device array of PIR_NOALLOC_SCRATCH_BYTES per GPU, held
 *   from library load to process exit.  The first call on a device looks up the
 *   array's device address; make it before any stream capture.  All calls share
 *   the array, so calls that overlap on the GPU race: serialize them.
 *   Limit: the result ([L*n][2B][D2] words) plus one chunk of query scratch must
 *   fit the array; D1 is folded in as many chunks as needed.  Requests whose
 *   result alone does not fit return PIR_ERR_ARG.
 *   Calls no cudaMalloc, cudaFree or other allocating routine.
 * Errors: PIR_ERR_HANDLE, PIR_ERR_ARG (B = 0, NULL or misaligned buffers, too
 * large for the scratch array), PIR_ERR_CUDA. */
#define PIR_NOALLOC_SCRATCH_BYTES (64u << 20)
pir_status_t pir_answer_noalloc(pir_db_t db, const uint32_t *queries, uint32_t B, uint32_t *responses,
                                void *stream);

/* Forward / inverse negacyclic NTT of `count` RNS polynomials [count][L][n] in
 * place, in device memory, asynchronously on stream (Sec. 2.3; single-kernel
 * on-chip NTT, Sec. 4.3).  Inputs must be canonical; outputs are canonical.
 * ntt_inv includes the scaling by n^-1, so ntt_inv(ntt_fwd(a)) = a.
 * Errors: PIR_ERR_ARG (NULL, misaligned, invalid params), PIR_ERR_CUDA. */
pir_status_t ntt_fwd(const pir_params_t *params, uint32_t *polys, size_t count, void *stream);
pir_status_t ntt_inv(const pir_params_t *params, uint32_t *polys, size_t count, void *stream);

/* Inverse NTT with modulus switching fused into it (Sec. 4.3 fuses the modulus
 * reduction into the inverse NTT; App. D.5, "Error analysis of RLWE modulus
 * switching", defines the switch from q = q_0 ... q_{L-1} to one prime).
 *   in:  [count][L][n] uint32, NTT form over q, canonical; device memory, read only.
 *   out: [count][n] uint32, coefficient form over q_0 (the first prime of params),
 *        canonical; device memory, written.  out[c][t] = round(x q_0 / q) mod q_0,
 *        x in [0, q) being the CRT lift of coefficient t of ntt_inv(in[c]).
 * Both buffers 16-byte aligned and disjoint; asynchronous on stream.  With L = 1 the
 * result equals ntt_inv.  Errors: PIR_ERR_ARG (NULL, misaligned or overlapping
 * buffers, invalid params), PIR_ERR_CUDA. */
pir_status_t ntt_inv_modswitch(const pir_params_t *params, const uint32_t *in, size_t count, uint32_t *out,
                               void *stream);

/* Server-side query expansion (Sec. 3.5, "ExpPack" expansion; App. C.2, SealPIR's
 * recursive expansion after pre-scaling by 2^-levels; App. D.3, expansion keys with
 * ell gadget digits of base t = 2^ceil(log2 q / ell)).  A client sends one packed
 * ciphertext per query, an encryption of m = sum_i m_i X^i, instead of D1
 * ciphertexts; the server expands it into D1 ciphertexts that each encrypt m_i as
 * a constant polynomial (a one-hot first-dimension query packs m = X^i*).
 *
 * pir_expander_create loads a client's expansion keys: keys[levels][ell][2][L][n]
 * uint32, coefficient form, canonical; key j switches from tau_g(s) to s for
 * g = n / 2^j + 1 (App. C.2's level j), key digit k is an encryption of t^k tau_g(s)
 * (a_k s + b_k = t^k tau_g(s) + e_k).  Host or device memory (keys_on_device); the
 * call copies them, turns them to NTT form and synchronizes `stream`.  levels is
 * the expansion depth (2^levels <= n; a DB needs 2^levels >= D1); ell the digit
 * count, with t = 2^w, w = ceil(ceil(log2 q) / ell) <= 30.  The handle owns device
 * memory until pir_expander_free.
 * Errors: PIR_ERR_ARG (NULL, invalid params, levels or ell out of range), PIR_ERR_OOM,
 * PIR_ERR_CUDA. */
typedef struct pir_expander *pir_expander_t;
pir_status_t pir_expander_create(const pir_params_t *params, uint32_t levels, uint32_t ell, const uint32_t *keys,
                                 int keys_on_device, void *stream, pir_expander_t *out);
pir_status_t pir_expander_free(pir_expander_t expander);

/* Expand B packed ciphertexts, packed [B][2][L][n] (coefficient form, canonical,
 * device memory), into out [B][count][2][L][n] (coefficient form, canonical, device
 * memory; count <= 2^levels): out[b][i] encrypts coefficient i of query b's packed
 * message.  Asynchronous on stream; scratch from the stream-ordered allocator.
 * Errors: PIR_ERR_HANDLE, PIR_ERR_ARG (NULL or misaligned buffers, B = 0, count out
 * of range), PIR_ERR_OOM, PIR_ERR_CUDA. */
pir_status_t pir_expand(pir_expander_t expander, const uint32_t *packed, uint32_t B, uint32_t count, uint32_t *out,
                        void *stream);

/* pir_answer for packed queries: expands packed [B][2][L][n] into the D1 query
 * ciphertexts of every query (in NTT form, on the device) and answers them; the
 * responses are those pir_answer_ex gives for the expanded queries, [B][D2][2][L][n]
 * (or [B][D2][2][n] with PIR_ANSWER_MODSWITCH).  on_device as for pir_answer.  opts
 * as for pir_answer_ex, except that k_chunk must be 0 or >= D1 (the expanded queries
 * are whole) and PIR_ANSWER_TEST_STALL is refused; with PIR_ANSWER_STAGE_TIMES the
 * expansion counts as stage 0.  The expander's ring must be the DB's.
 * Errors: PIR_ERR_HANDLE, PIR_ERR_ARG (mismatched ring, 2^levels < D1, bad buffers or
 * options), PIR_ERR_UNSUPPORTED (limb layout with D1 not a multiple of 32 or above
 * 8192), PIR_ERR_OOM, PIR_ERR_CUDA. */
pir_status_t pir_answer_packed(pir_db_t db, pir_expander_t expander, const uint32_t *packed, uint32_t B,
                               uint32_t *responses, int on_device, void *stream, const pir_answer_opts_t *opts);

/* pir_graph_create for packed queries (pir_answer_packed below, device buffers):
 * the expansion and the answer captured together, so that the expansion's many
 * small launches (about 36 at batch 1 on the 1 GiB DB) replay without launch gaps.
 * The graph reads the expander's keys: freeing the expander (or the DB) makes
 * pir_graph_launch refuse the graph with PIR_ERR_HANDLE.  packed [B][2][L][n] and
 * responses as for pir_answer_packed; opts: k_chunk 0 (or >= D1), tile, and
 * PIR_ANSWER_MODSWITCH.  The paper has no counterpart (a launch mechanism).
 * Errors: PIR_ERR_HANDLE, PIR_ERR_ARG, PIR_ERR_OOM, PIR_ERR_CUDA. */
pir_status_t pir_graph_create_packed(pir_db_t db, pir_expander_t expander, const uint32_t *packed, uint32_t B,
                                     uint32_t *responses, const pir_answer_opts_t *opts, pir_graph_t *out);

/* Folding of the remaining dimensions with RGSW-RLWE external products (Sec. 3.2 and
 * 3.6: OnionPIR's construction; gadget of App. D.3).  Each level pairs the
 * ciphertexts (2j, 2j+1) of a query and keeps c_2j + RGSW_l (x) (c_2j+1 - c_2j), where
 * the external product writes both components of the difference in the gadget (ell
 * digits of base t = 2^w, w = ceil(ceil(log2 q) / ell) <= 30, of the CRT lift of every
 * coefficient) and sums digit x row products.  RGSW_l encrypting the bit l of the
 * wanted index selects that ciphertext.  An RGSW ciphertext is 2 ell RLWE rows: row
 * k < ell encrypts zero plus mu t^k in its a-part, row ell + k zero plus mu t^k in its
 * b-part.
 *   pir_fold: cts [B][2^levels][2][L][n] -> out [B][2][L][n]; rgsw
 *     [B][levels][2 ell][2][L][n]; all coefficient form, canonical, device memory,
 *     16-byte aligned; asynchronous on stream.
 *   pir_answer_folded: the first-dimension answer of pir_answer_ex (queries
 *     [B][D1][2][L][n]) folded over all log2(D2) remaining levels (D2 a power of two)
 *     with rgsw [B][log2 D2][2 ell][2][L][n]: responses [B][2][L][n], or [B][2][n] over
 *     q_0 with PIR_ANSWER_MODSWITCH; one ciphertext per query holding the record.
 *     on_device and opts as for pir_answer_ex (PIR_ANSWER_TEST_STALL refused; with
 *     PIR_ANSWER_STAGE_TIMES the folding and the final inverse NTT count as stage 4).
 * Errors: PIR_ERR_HANDLE, PIR_ERR_ARG (NULL or misaligned buffers, B = 0, ell out of
 * range or digits above 30 bits, D2 not a power of two), PIR_ERR_OOM, PIR_ERR_CUDA. */
pir_status_t pir_fold(const pir_params_t *params, const uint32_t *cts, uint32_t B, uint32_t levels, uint32_t ell,
                      const uint32_t *rgsw, uint32_t *out, void *stream);
pir_status_t pir_answer_folded(pir_db_t db, const uint32_t *queries, uint32_t B, uint32_t ell, const uint32_t *rgsw,
                               uint32_t *responses, int on_device, void *stream, const pir_answer_opts_t *opts);

/* Scalar-HE (LWE) DB GEMM of SimplePIR's online step (Sec. 2.5), built as Sec. 4.1
 * builds it on the INT8 tensor pipe:
 *     out[b][i] = sum_j db[i][j] * queries[b][j]   (mod 2^32)
 *   db:      [D1][D0] int8 (signed plaintexts; the raw DB, no encoding), device.
 *   queries: [B][D0] uint32 (the query ciphertexts' Z_2^32 entries), device.
 *   out:     [B][D1] uint32, device, written.
 * Each query word is split into four byte planes (prmt), each plane multiplied on
 * the tensor pipe (mma.sync s8 x u8 -> s32, wrapping = mod 2^32) and the planes
 * recombined by shifts.  path: PIR_LWE_TENSOR, PIR_LWE_SIMT (CUDA-core dp4a on the
 * same byte planes), or PIR_LWE_AUTO (tensor from 8 queries up).  D0 must be a
 * multiple of 16 and at most 2^24; buffers 16-byte aligned.  Asynchronous on
 * stream; the caller owns every buffer.
 * Errors: PIR_ERR_ARG (NULL or misaligned buffers, zero or unsupported sizes, unknown
 * path), PIR_ERR_CUDA. */
#define PIR_LWE_AUTO 0u
#define PIR_LWE_TENSOR 1u
#define PIR_LWE_SIMT 2u
pir_status_t pir_lwe_answer(const int8_t *db, uint32_t D1, uint32_t D0, const uint32_t *queries, uint32_t B,
                            uint32_t *out, uint32_t path, void *stream);

/* Measured peak of the INT8 warp-level tensor instruction (mma.sync m16n8k32 s8 x u8
 * -> s32) on the current device, in tera-operations per second (2 per multiply-add):
 * the denominator of the scalar-HE GEMM's roofline.  The paper has no counterpart.
 * Synchronizes `stream`.  Errors: PIR_ERR_ARG (NULL), PIR_ERR_CUDA. */
pir_status_t pir_probe_int8_mma(void *stream, double *tops);
/* Release a DB handle and its device memory (synchronizes the device first). */
pir_status_t pir_free_db(pir_db_t db);

/* Resident device bytes of a DB. */
pir_status_t pir_db_bytes(pir_db_t db, size_t *bytes);

/* The parameters and layout a DB was set up with. */
pir_status_t pir_db_info(pir_db_t db, pir_params_t *params, int *layout);

/* Copy the NTT-form residues of DB polynomial (i, c) = poly_index / D2, % D2 to
 * host memory out[L][n] (canonical, NTT order as above).  For inspection and
 * tests; synchronous. */
pir_status_t pir_db_read_poly(pir_db_t db, uint64_t poly_index, uint32_t *out);

/* Human-readable name of a status; never NULL. */
const char *pir_status_str(pir_status_t status);

/* The last CUDA error string seen by this library on the calling thread ("" if none). */
const char *pir_last_cuda_error(void);

/* Number of GEMM tile choices for a layout (ids 1..count for pir_answer_opts_t.tile). */
uint32_t pir_gemm_tiles(int layout);

/* Per-stage device time of the answers issued with PIR_ANSWER_STAGE_TIMES by the
 * calling thread since the last reset: waits for their events, adds each stage's
 * elapsed milliseconds into ms[PIR_STAGES] and its kernel launches into
 * launches[PIR_STAGES] (either may be NULL), and resets.  The events are recorded on
 * the stream each stage runs on, so a stage's time is its kernels' time on that
 * stream.  Errors: PIR_ERR_CUDA. */
pir_status_t pir_stage_times(double *ms, uint64_t *launches);

/* Number of kernels this library has launched in this process (all threads). */
uint64_t pir_kernel_launches(void);

/* The library keeps freed answer scratch cached in the current device's
 * stream-ordered memory pool (repeated answers then allocate nothing new) and
 * graph scratch in its graph memory pool.  This call gives all of it that no work
 * in flight uses back to the device, for allocations made outside the library.
 * The library does the same by itself before it refuses an allocation, a graph
 * launch or a DB.  Errors: PIR_ERR_CUDA. */
pir_status_t pir_release_memory(void);

/* Kernels that wait on barriers (the TMA-staged scan) bound every wait to about
 * one second; a wait that runs out sets a per-device error word, the kernel
 * drains its copies in flight and returns early (its output is then invalid).
 * This call synchronizes `stream`, reads and clears the current device's word and
 * returns PIR_ERR_TIMEOUT if it was set, else PIR_OK. */
pir_status_t pir_check_device(void *stream);

/* The same device error word read without waiting for any work: the copy runs on a
 * stream of the library's own that nothing else uses, so kernels still running (a
 * batch that never completes included) do not hold it up.  Reads and clears the
 * current device's word; returns PIR_ERR_TIMEOUT if it was set, else PIR_OK (a
 * wait that runs out while the read is in flight shows in the next read).
 * Errors: PIR_ERR_CUDA. */
pir_status_t pir_device_status(void);

#ifdef __cplusplus
}
#endif
#endif /* GBPIR_H */
