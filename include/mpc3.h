/*
 * libmpc3 -- maliciously secure three-party linear-function evaluation over Z_2^64 on one GPU.
 *
 * The library implements the hot path of "The Communication-Friendly Privacy-Preserving Machine
 * Learning against Malicious Adversaries" (arXiv 2411.09287): the <.>-sharing of Sec. 2, Pi_Mult
 * (Fig. MultP), Pi_Inner for matrix products (Fig. DPP, Sec. 4.1), Pi_Trunc (Fig. trunc), the
 * batched verification Pi_MultVerify / Pi_BIVerify (Fig. PPEV, Fig. PBDP) built from Pi_Tran
 * (Fig. MTP), Pi_Reduce (Fig. Reduce) and Pi_InnerVerify (Fig. DPV) over GR(2^64, 64), and
 * Pi_Rec (Sec. 2).  All three parties P0, P1, P2 are simulated on one GPU: each holds its own
 * device copy of every share it owns, and every protocol message is a device-to-device copy that
 * is counted in a ledger.
 *
 * Conventions
 *   - All values are uint64_t, i.e. elements of Z_2^64; arithmetic wraps mod 2^64.
 *   - A <.>-shared tensor of n elements ("sharing") is one device buffer of 6*n words, component c
 *     at [c*n, (c+1)*n):  0: P0.[r]_1  1: P0.[r]_2  2: P1.m  3: P1.[r]_1  4: P2.m  5: P2.[r]_2,
 *     with m = x + [r]_1 + [r]_2 (Sec. 2 Notation).  Matrices are row-major inside a component.
 *   - Every call enqueues work on the context's stream and returns once it is enqueued, except
 *     mpc_verify_* and mpc_reconstruct with a host output, which synchronise to read the result.
 *   - Buffers passed in are borrowed for the duration of the enqueued work; the caller owns them.
 *     `workspace` is caller-owned device scratch of at least mpc_workspace_size(...) bytes,
 *     256-byte aligned; its contents are undefined after the call.
 *   - call_id / verify_id name the PRG streams of a call (< 2^44).  Two calls must not share an
 *     id.  Randomness is drawn from ChaCha20 (RFC 8439) keyed per party pair from the seed.
 *   - Return value: MPC_OK or one of the MPC_ERR_* codes below; mpc_last_error() describes the
 *     last failure.  After MPC_ERR_ABORT or MPC_ERR_VERIFY the context is aborted (security with
 *     abort, Sec. 2 "Security Model") and every later call returns MPC_ERR_ABORT.
 */
#ifndef MPC3_H
#define MPC3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPC3_ABI_VERSION 1

enum {
  MPC_OK = 0,
  MPC_ERR_ARG = 1,        /* invalid argument (null pointer, bad id, bad enum)              */
  MPC_ERR_SHAPE = 2,      /* invalid sizes                                                   */
  MPC_ERR_WORKSPACE = 3,  /* workspace smaller than mpc_workspace_size()                     */
  MPC_ERR_CUDA = 4,       /* a CUDA call failed (message in mpc_last_error)                  */
  MPC_ERR_TIMEOUT = 5,    /* a bounded device wait expired (the context aborts)              */
  MPC_ERR_VERIFY = 6,     /* the batched check found Delta != 0 (Fig. DPV outputs 0)         */
  MPC_ERR_ABORT = 7,      /* Pi_Rec saw inconsistent messages, or the context is aborted     */
  MPC_ERR_PENDING = 8     /* reconstruction requested while products are unverified          */
};

/* third interpolation point of Pi_Reduce (Fig. Reduce), whose interpolation at 0, 1, 2 divides by 2
 * (not a unit of GR(2^64, 64)): POINT_X interpolates at 0, 1, x (x the ring generator; x and
 * 1 - x are units) for any challenge; POINT_2 keeps 0, 1, 2 and evaluates at zeta = 2 zeta' so
 * that the Lagrange weights stay integral */
enum { MPC_REDUCE_POINT_X = 0, MPC_REDUCE_POINT_2 = 1 };
/* local products of Pi_Inner: exact u64 CUDA-core GEMM, or exact limb-split tensor-core GEMM */
enum { MPC_GEMM_U64 = 0, MPC_GEMM_LIMB_TC = 1 };
/* ledger axes */
enum { MPC_PHASE_OFFLINE = 0, MPC_PHASE_ONLINE = 1, MPC_PHASE_VERIFY = 2, MPC_NPHASE = 3 };
enum {
  MPC_PROTO_SHARE = 0, MPC_PROTO_MULT = 1, MPC_PROTO_INNER = 2, MPC_PROTO_TRUNC = 3,
  MPC_PROTO_REC = 4, MPC_PROTO_VERIFY = 5, MPC_NPROTO = 6
};
/* host-side fault injection sites (a cheating sender corrupts one delivered element) */
enum {
  MPC_SITE_GAMMA2 = 0,      /* P0 -> P2 [Gamma]_2 of Pi_Mult / Pi_Inner / trunc pairs        */
  MPC_SITE_MZ1 = 1,         /* P1 -> P2 [m_z]_1                                              */
  MPC_SITE_MZ2 = 2,         /* P2 -> P1 [m_z]_2                                              */
  MPC_SITE_MX_COPY_P1 = 3,  /* P0 -> P1 m of an input sharing (inconsistent replica)         */
  MPC_SITE_REC_MSG = 4,     /* P0 -> P1 [r]_2 of Pi_Rec                                      */
  MPC_SITE_HIGH_BIT = 5,    /* [Gamma]_2 XOR 2^63: the ring attack of Sec. 3                 */
  MPC_SITE_AND_GAMMA2 = 6,  /* P0 -> P2 [Gamma]_2 of a Boolean AND gate (non-linear layers):
                               flips bit `index` of the packed message when mask & 1            */
  MPC_SITE_TRUNC_D1 = 7,    /* P1 -> P2 mask-switch message d1 of mpc_trunc                   */
  MPC_NSITE = 8
};
/* workspace queries */
enum {
  MPC_OP_SHARE = 0, MPC_OP_MULT = 1, MPC_OP_MATMUL = 2, MPC_OP_VERIFY_MULT = 3,
  MPC_OP_VERIFY_MATMUL = 4, MPC_OP_RECONSTRUCT = 5, MPC_OP_RELU = 6, MPC_OP_MAXPOOL2 = 7,
  MPC_OP_VERIFY_MULT_CALLS = 8, MPC_OP_SHARE_FIXED = 9, MPC_OP_RECONSTRUCT_FIXED = 10,
  MPC_OP_TRUNC = 11, MPC_OP_VERIFY_TRUNC = 12
};

typedef struct mpc_ctx mpc_ctx;

typedef struct {
  uint8_t seed[32];   /* master seed; pair keys eta01, eta02, eta12 are derived from it        */
  int device;         /* CUDA device ordinal                                                    */
  int reduce_mode;    /* MPC_REDUCE_POINT_X (default) or MPC_REDUCE_POINT_2                     */
  int gemm_path;      /* MPC_GEMM_U64 or MPC_GEMM_LIMB_TC                                       */
  void* stream;       /* cudaStream_t to run on; NULL: the library creates its own              */
} mpc_config;

/* Tuning of the verification's data layout and of the tensor-core launches.  No setting changes
 * a protocol value: every one gives the same messages, revealed challenges, transcript and result
 * (the parity tests compare several with the oracle).  They trade workspace against time, let an
 * autotuner pick launch shapes, and let small problems take the code paths that only large ones
 * take by default.  A field left 0 keeps its default; mpc_get_tuning returns resolved values.
 *   trunc_block    L, the block of the truncation batch's weights r^(2e), e = e_hi L + e_lo (Fig.
 *                  PBDP weights, Fig. trunc pairs): a batch of E >= L outputs is blocked, its
 *                  S-matrix inner sums run per block and, when E is a multiple of L on the
 *                  tensor-core path, only the first block of powers is kept.  Multiple of 128,
 *                  at most 65536 (the S-matrix kernel's exactness bound); default 65536.
 *   trunc_chunk    most outputs per verification chunk of the truncation batch (see
 *                  mpc_verify_matmul); at least 1; default 2^24.
 *   row_split      L', rows per block of the blocked batch's folded-vector products
 *                  (x_e = r^(2 L' e_hi) sum_j b_(e,j) r^(2 e_lo) V_j, e = e_hi L' + e_lo);
 *                  multiple of 128; default: the odd multiple of 128 near sqrt(E) that pads least.
 *                  A batch uses at most E rounded up to a multiple of 128; a row_split above
 *                  trunc_block keeps the whole table of powers (no compact table).
 *   tc_combine_min fewest e_hi blocks for which sum_(e_hi) r^(2 L e_hi) S_hi runs on the tensor
 *                  cores (fewer: CUDA cores); default 32.
 *   gemm_split_min fewest 32-deep K chunks per split-K slice of a thin tensor-core product;
 *                  default 8.
 *   gram_split     split-K slices of a tensor-core Gram sum (dense rounds); default 76.
 *   fold_batch_max the folds of one Pi_Reduce round share one launch when the folded vectors
 *                  have at most this many elements; default 65536.
 *   gr_producers   how the GR-matrix products (folds, tables) load their A rows: 1 producer
 *                  warps' global loads into registers (two digit-plane stages), 2 TMA loads of
 *                  half-chunks into shared memory (one digit-plane stage, rewritten by K halves
 *                  as the MMAs of each half finish), 3 TMA loads with the A digit planes in
 *                  tensor memory (output in two halves of 32 columns); default 2.
 *   gr_drain_warps warps that drain the GR-matrix products' accumulators: 8 or 16; default 8. */
typedef struct {
  int64_t trunc_block;
  int64_t trunc_chunk;
  int64_t row_split;
  int32_t tc_combine_min;
  int32_t gemm_split_min;
  int32_t gram_split;
  int32_t fold_batch_max;
  int32_t gr_producers;
  int32_t gr_drain_warps;
} mpc_tuning;

/* Create a context (keys, stream, device constants, ledger).  *out is NULL on failure. */
int mpc_create(const mpc_config* cfg, mpc_ctx** out);
/* Destroy a context; waits for its work.  NULL is ignored. */
void mpc_destroy(mpc_ctx* ctx);
/* Description of the last failure of this context ("" if none).  Owned by the context. */
const char* mpc_last_error(const mpc_ctx* ctx);
/* ---- asynchronous copies ---------------------------------------------------------------------
 * A pipelined caller uploads the next step's inputs and downloads the last step's result while
 * the current step runs:
 *   mpc_h2d_async copies `bytes` from host `src` (pinned memory, for the copy to overlap) to
 *     device `dst` on the context's copy stream (created on first use), after the work enqueued
 *     so far on the context's stream (which may still read `dst`); it overlaps the work enqueued
 *     after it, so step k + 1's upload is issued before step k is enqueued;
 *   mpc_d2h_async copies `bytes` from device `src` to host `dst` (pinned) on the copy stream,
 *     after the work enqueued so far on the context's stream (which writes `src`);
 * each records the copy under `slot` (0 .. MPC_H2D_SLOTS - 1).  mpc_h2d_wait makes the context's
 * stream wait, on the device, for the copy last recorded under `slot` (no host synchronisation; a
 * slot never used is a no-op): before work that reads an uploaded buffer, or that rewrites a
 * buffer still being downloaded.  A download is complete on the host after a device
 * synchronisation.  The caller owns all buffers.
 * Returns MPC_OK, MPC_ERR_ARG (null pointer, zero bytes, bad slot) or MPC_ERR_CUDA. */
#define MPC_H2D_SLOTS 4
int mpc_h2d_async(mpc_ctx* ctx, void* dst, const void* src, size_t bytes, int slot);
int mpc_d2h_async(mpc_ctx* ctx, void* dst, const void* src, size_t bytes, int slot);
int mpc_h2d_wait(mpc_ctx* ctx, int slot);

/* Run subsequent work on `stream` (cudaStream_t). */
int mpc_set_stream(mpc_ctx* ctx, void* stream);
/* Replace the context's tuning (NULL: all defaults).  MPC_ERR_ARG for a value out of range
 * (negative, or trunc_block / row_split not a multiple of 128, trunc_block > 65536).  Workspace
 * sizes depend on the tuning: query mpc_workspace_size after setting it. */
int mpc_set_tuning(mpc_ctx* ctx, const mpc_tuning* tune);
/* The tuning in force, defaults resolved (row_split 0 means: chosen per batch). */
int mpc_get_tuning(const mpc_ctx* ctx, mpc_tuning* out);
/* Wait for all enqueued work; returns MPC_ERR_CUDA on an asynchronous CUDA error. */
int mpc_sync(mpc_ctx* ctx);
/* MPC_OK, or MPC_ERR_ABORT once the context has aborted. */
int mpc_status(const mpc_ctx* ctx);

/* Bytes of workspace an operation needs.  op = MPC_OP_*; (a, b, c) = (n, 0, 0) for SHARE, MULT,
 * VERIFY_MULT, RECONSTRUCT, RELU, SHARE_FIXED, RECONSTRUCT_FIXED, TRUNC and VERIFY_TRUNC, (total n
 * of all calls, 0, 0) for VERIFY_MULT_CALLS, (M, N, K) for MATMUL and VERIFY_MATMUL (a
 * convolution: M = B Ho Wo, N = C_out, K = C kh kw), (B C, H, W) for MAXPOOL2; trunc_bits, R_main
 * and R_trunc as passed to the operation (R < 0: default; VERIFY_MULT and VERIFY_MULT_CALLS take
 * their R in R_main, VERIFY_TRUNC in R_trunc).  Returns -1 for invalid arguments. */
int64_t mpc_workspace_size(const mpc_ctx* ctx, int op, int64_t a, int64_t b, int64_t c,
                           int trunc_bits, int R_main, int R_trunc);

/* Pi_<.>^{l,0}(x) (Sec. 2, Secret sharing, owner P0): [r_x]_1 from eta01, [r_x]_2 from eta02,
 * and P0 sends m_x = x + [r_x]_1 + [r_x]_2 to P1 and P2 (2 l bits per element).
 * x: n plaintext words, on the host if x_on_host (copied in, stream-ordered) else on the device.
 * xs: device sharing (6n words) written by the call. */
int mpc_share_input(mpc_ctx* ctx, uint64_t call_id, const uint64_t* x, int x_on_host, int64_t n,
                    uint64_t* xs, void* workspace, size_t workspace_bytes);

/* Pi_<.>^{l,k}(x) (Sec. 2, Secret sharing) for an input owned by P_k, k in {0, 1, 2}.  The owner
 * holds both seeds of the input's mask, so the sharing equals mpc_share_input's for the same
 * call_id; only the messages differ.  k = 0 is mpc_share_input: P0 sends m_x to P1 and P2, 2 l
 * bits per element.  k = 1 (2) keeps its own copy of m_x and sends m_x to P2 (P1), l bits per
 * element.  Arguments, workspace (MPC_OP_SHARE) and return codes as mpc_share_input;
 * MPC_ERR_ARG for another owner. */
int mpc_share_input_from(mpc_ctx* ctx, uint64_t call_id, int owner, const uint64_t* x,
                         int x_on_host, int64_t n, uint64_t* xs, void* workspace,
                         size_t workspace_bytes);

/* Pi_Mult (Fig. MultP), elementwise z_i = x_i y_i: preprocessing ([r_z] <- Pi_[.]; P0 shares
 * Gamma = r_x r_y + r_z, 1 l bits) and online phase (P1, P2 exchange [m_z]_j, 2 l bits).
 * xs, ys: device sharings of n elements; zs: device sharing written by the call.  The triples
 * stay pending until mpc_verify_mult(..., mult_call_id = call_id, ...). */
int mpc_mult(mpc_ctx* ctx, uint64_t call_id, const uint64_t* xs, const uint64_t* ys, int64_t n,
             uint64_t* zs, void* workspace, size_t workspace_bytes);

/* Pi_Inner for every output of Z = X W (Fig. DPP; Sec. 4.1 views an M x N product as M N inner
 * products of dimension K), X: M x K, W: K x N.  With trunc_bits = t >= 0 also Pi_Trunc^t
 * (Fig. trunc): the product wire's mask is the truncation pair's r_x, and the output
 * zout has m = m_Z >>_arith t and mask r_z = r_x >>_arith t (communication 7 l offline, 2 l
 * online per output, Table 1).  With trunc_bits < 0, zout may equal zpre or be NULL and pq is
 * ignored.
 *   xs: 6 M K words; ws_: 6 K N words; zpre, zout: 6 M N words each (written);
 *   pq: 12 M N words (written): the sharings <p> and <q> of the trunc pair's two inner products,
 *       kept for mpc_verify_matmul. */
int mpc_matmul(mpc_ctx* ctx, uint64_t call_id, const uint64_t* xs, const uint64_t* ws_,
               int64_t M, int64_t N, int64_t K, int trunc_bits, uint64_t* zpre, uint64_t* zout,
               uint64_t* pq, void* workspace, size_t workspace_bytes);

/* mpc_matmul with the truncation pairs' random bits keyed by output row: the bits b1, b2 of output
 * (a, b) are word b of the bit streams of object row_keys[a] (instead of word a N + b of the
 * call's streams).  Every other random value stays the call's.  A truncated output's opened value
 * depends on the other party-random values only through its pair mask r_x = b1 xor b2 (the carry
 * of Fig. trunc), so rows keyed by (request, layer, row of the request) open to the same values
 * whichever batch they are packed into; serving uses this to return a request the same logits
 * alone and packed.  row_keys: M device words (borrowed), object ids as call_id << 20 | batch << 16
 * | sub with call_id < 2^44; NULL is mpc_matmul.  Verify with mpc_verify_matmul_keyed and the
 * same keys. */
int mpc_matmul_keyed(mpc_ctx* ctx, uint64_t call_id, const uint64_t* xs, const uint64_t* ws_,
                     int64_t M, int64_t N, int64_t K, int trunc_bits, const uint64_t* row_keys,
                     uint64_t* zpre, uint64_t* zout, uint64_t* pq, void* workspace,
                     size_t workspace_bytes);

/* Pi_MultVerify^R (Fig. PPEV) of the n triples (x_i, y_i, z_i) produced by
 * mpc_mult(call_id = mult_call_id): Pi_Tran with a revealed challenge r, R rounds of Pi_Reduce,
 * then Pi_InnerVerify.  R < 0 selects max(0, ceil(log2 n) - 6).  Returns MPC_OK if the check
 * accepts, MPC_ERR_VERIFY if Delta != 0, MPC_ERR_ABORT if a Pi_Rec inside aborted.
 * trace (device, optional): per round k = 1..R at offset (k-1)*832 the revealed zeta' (64 words),
 * <h(0)> (6 x 64), <h(p2)> (6 x 64); then the opened Delta (64) at R*832. */
int mpc_verify_mult(mpc_ctx* ctx, uint64_t verify_id, const uint64_t* xs, const uint64_t* ys,
                    const uint64_t* zs, int64_t n, uint64_t mult_call_id, int R,
                    void* workspace, size_t workspace_bytes, uint64_t* trace);

/* Deferred Pi_MultVerify^R (Fig. PPEV) of the triples of several mpc_mult calls in one batch, e.g.
 * every gate of a multiplication circuit checked once before any output is opened (outputs are
 * reconstructed only after verification, Sec. 2).  Call l produced the n[l] triples (xs[l], ys[l],
 * zs[l]) under call id call_ids[l]; the batch is their concatenation in the order given, so the
 * transcript equals that of mpc_verify_mult on the concatenated sharings (component c of call l at
 * offset n[0] + ... + n[l-1] of component c).  xs, ys, zs: host arrays of ncalls device pointers,
 * each a sharing of 6 n[l] words; n, call_ids: host arrays of ncalls entries, read during the
 * call only.  Workspace: mpc_workspace_size(MPC_OP_VERIFY_MULT_CALLS, n[0] + ... + n[ncalls-1],
 * 0, 0, -1, R, -1).  Every listed call leaves the pending state once the check has accepted (a
 * rejection makes the context abort).  R < 0 selects max(0, ceil(log2 N) - 6) for the total N.
 * Returns as mpc_verify_mult; MPC_ERR_ARG / MPC_ERR_SHAPE for a null pointer, a bad id, a call
 * id that is not a pending mpc_mult call or is listed twice, or n[l] <= 0.  trace: as
 * mpc_verify_mult. */
int mpc_verify_mult_calls(mpc_ctx* ctx, uint64_t verify_id, int ncalls,
                          const uint64_t* const* xs, const uint64_t* const* ys,
                          const uint64_t* const* zs, const int64_t* n, const uint64_t* call_ids,
                          int R, void* workspace, size_t workspace_bytes, uint64_t* trace);

/* Pi_BIVerify (Fig. PBDP) of the layer produced by mpc_matmul(call_id = matmul_call_id):
 * batch 0 = the M N inner products of Z = X W, consolidated with weights r^(aN+b) and evaluated
 * as the K-dimensional claim sum_k Xt_k Wt_k = zt (rank-1 form: Xt = X^T P, Wt = W Q with P, Q
 * the weight powers); batch 1 (when trunc_bits >= 0) = the 2 M N inner products of the truncation
 * pairs, merged per output into one 64-dimensional inner product.  Batch 1 is checked in chunks
 * of at most tuning.trunc_chunk consecutive outputs (row-major e = aN + b): chunk i covers
 * outputs [i C, min(E, (i + 1) C)) and is a batch of its own, with its own challenge r (the
 * streams of batch 1 + i), weights r^(2e') over the chunk-local index e' and its own rounds
 * (reading of Fig. PBDP: a layer's inner products may be split into independently verified
 * batches; chunk i is sound up to |G_i| / 2^(d - R_i - 2), Thm. multvv).  At most 15 chunks, else
 * MPC_ERR_SHAPE.  R_main / R_trunc < 0 select the default max(0, ceil(log2 D) - 6) (D = 64 E_i
 * per chunk).  Returns as mpc_verify_mult.  trace (device, optional; mpc_trace_words words):
 * batch 0 as in mpc_verify_mult, then each chunk's R_i + 1 blocks in chunk order. */
int mpc_verify_matmul(mpc_ctx* ctx, uint64_t verify_id, const uint64_t* xs, const uint64_t* ws_,
                      const uint64_t* zpre, const uint64_t* pq, int64_t M, int64_t N, int64_t K,
                      int trunc_bits, uint64_t matmul_call_id, int R_main, int R_trunc,
                      void* workspace, size_t workspace_bytes, uint64_t* trace);

/* mpc_verify_matmul (Fig. PBDP, Fig. trunc) of a layer made by mpc_matmul_keyed (reading A12):
 * the truncation batch regenerates the pairs' bits from the same row keys (M device words; NULL
 * is mpc_verify_matmul). */
int mpc_verify_matmul_keyed(mpc_ctx* ctx, uint64_t verify_id, const uint64_t* xs,
                            const uint64_t* ws_, const uint64_t* zpre, const uint64_t* pq,
                            int64_t M, int64_t N, int64_t K, int trunc_bits,
                            const uint64_t* row_keys, uint64_t matmul_call_id, int R_main,
                            int R_trunc, void* workspace, size_t workspace_bytes,
                            uint64_t* trace);

/* Words of the optional verification trace of op = MPC_OP_VERIFY_MULT, MPC_OP_VERIFY_MULT_CALLS,
 * MPC_OP_VERIFY_MATMUL or MPC_OP_VERIFY_TRUNC, arguments as mpc_workspace_size; -1 for invalid
 * arguments. */
int64_t mpc_trace_words(const mpc_ctx* ctx, int op, int64_t a, int64_t b, int64_t c,
                        int trunc_bits, int R_main, int R_trunc);

/* Pi_Rec (Sec. 2): P0 sends [r]_1 to P2 and [r]_2 to P1, P1 sends m to P0; P1 sends H([r]_1) to
 * P2, P2 sends H(m) to P0 and H([r]_2) to P1 (H = SHA-256 Merkle root, 1 KiB leaves).  On any
 * mismatch the call returns MPC_ERR_ABORT; otherwise out = m - [r]_1 - [r]_2 (n words, host if
 * out_on_host, else device).  Refused with MPC_ERR_PENDING while products are unverified. */
int mpc_reconstruct(mpc_ctx* ctx, const uint64_t* xs, int64_t n, uint64_t* out, int out_on_host,
                    void* workspace, size_t workspace_bytes);

/* Pi_Rec (Sec. 2) without any device allocation: the same protocol, messages, checks and result as
 * mpc_reconstruct with a device output, but the received shares and the hash scratch live in
 * one fixed device array compiled into the library instead of a caller-provided workspace.  The
 * paper has no counterpart; this serves callers that cannot allocate device memory when they
 * reconstruct (a process whose free device memory is all held by its own pool, or a loop that
 * must not call cudaMalloc/cudaFree because they may synchronise the device).
 *   n: 1 .. MPC_NOALLOC_MAX_N elements, else MPC_ERR_SHAPE; out: n device words (written).
 *   The array costs about 6 MiB on every GPU that loads the library, for the life of the
 *   process.  The first call on a device resolves the array's address there; make that first
 *   call before any stream capture.  All calls share the array, so calls that can overlap on the
 *   GPU (other streams or contexts on the same device) race and must be serialised.
 *   Returns MPC_ERR_ABORT on inconsistent messages, MPC_ERR_PENDING while products are
 *   unverified. */
#define MPC_NOALLOC_MAX_N 262144
int mpc_reconstruct_noalloc(mpc_ctx* ctx, const uint64_t* xs, int64_t n, uint64_t* out);

/* Fixed-point input sharing (Sec. 2 Notation: x is encoded as floor(x 2^k) mod 2^l, two's
 * complement for x < 0), then Pi_<.>^{l,k}(x) exactly as mpc_share_input_from (owner 0, 1 or 2).
 * x 2^k outside [-2^63, 2^63) saturates to the nearest end and NaN encodes 0 (the paper assumes
 * values in range).  x: n doubles, on the host if x_on_host (copied in; the call then waits for
 * the copy, so x may be reused on return) else on the device; frac_bits: k in 0 .. 62.
 * Workspace: MPC_OP_SHARE_FIXED.  Returns as mpc_share_input. */
int mpc_share_fixed(mpc_ctx* ctx, uint64_t call_id, int owner, const double* x, int x_on_host,
                    int64_t n, int frac_bits, uint64_t* xs, void* workspace,
                    size_t workspace_bytes);

/* Pi_Rec (as mpc_reconstruct), then the fixed-point decoding of Sec. 2 Notation: out[i] = the
 * opened word read as a signed 64-bit integer, divided by 2^k.  out: n doubles, host if
 * out_on_host (the call waits for them) else device.  Workspace: MPC_OP_RECONSTRUCT_FIXED.
 * Returns as mpc_reconstruct (out is zeroed on an abort when it is on the host). */
int mpc_reconstruct_fixed(mpc_ctx* ctx, const uint64_t* xs, int64_t n, int frac_bits, double* out,
                          int out_on_host, void* workspace, size_t workspace_bytes);

/* A convolution as one Pi_Inner per output (Sec. 4.1: an m-dimensional convolution output is m
 * separate inner products), with Pi_Trunc^t when trunc_bits >= 0.  The library lowers the input
 * to the im2col rows of those inner products, then runs mpc_matmul on them:
 *   geom = {B, C, H, W, kh, kw, stride, pad}: xs is the NCHW sharing of B images of C x H x W;
 *   the kh x kw kernel moves by `stride` over the image padded with `pad` zeros on every side,
 *   Ho = (H + 2 pad - kh) / stride + 1 rows and Wo likewise;
 *   ws_: sharing of the (C kh kw) x C_out weight matrix, row (c, di, dj) = (c kh + di) kw + dj;
 *   cols (written): the 6 (B Ho Wo) (C kh kw)-word sharing of the lowered input, row
 *   (b, i, j) = (b Ho + i) Wo + j holding x[b][c][i stride + di - pad][j stride + dj - pad] (0 in
 *   the padding); keep it for the verification, which is mpc_verify_matmul(xs = cols, ws_, zpre,
 *   pq, B Ho Wo, C_out, C kh kw, trunc_bits, call_id, ...);
 *   zpre, zout, pq as mpc_matmul with M = B Ho Wo, N = C_out, K = C kh kw: output row (b, i, j),
 *   column c_out (NHWC order);
 *   row_keys: NULL, or M device words keying the truncation bits by output row as
 *   mpc_matmul_keyed does (verify with mpc_verify_matmul_keyed and the same keys).
 * Workspace: MPC_OP_MATMUL with (M, N, K) above.  MPC_ERR_SHAPE for a bad geometry. */
int mpc_conv2d(mpc_ctx* ctx, uint64_t call_id, const uint64_t* xs, const uint64_t* ws_,
               const int32_t geom[8], int64_t C_out, int trunc_bits, const uint64_t* row_keys,
               uint64_t* cols, uint64_t* zpre, uint64_t* zout, uint64_t* pq, void* workspace,
               size_t workspace_bytes);

/* Pi_Trunc^t (Fig. trunc) of a sharing <x> of n elements: <z> with z = x >>_arith t, up to the
 * one-LSB carry and the wrap of probability about |x| / 2^l that the paper states (Sec. 4.2).
 * Preprocessing as in Fig. trunc: the pairs (r_x, r_z = r_x >>_arith t) from 2 x 64 random bits
 * per element and two Pi_Inner of dimension 64 (6 l bits offline).  Fig. trunc assigns r_x to
 * the input wire before the gate that produces it runs (mpc_matmul does); x here was produced
 * with another mask r, so its mask is switched first: P1 sends d1 = [r_x]_1 - [r]_1 to P2, P2
 * sends d2 = [r_x]_2 - [r]_2 to P1 (2 l bits online), P0, who knows both, sends H(d1) to P2 and
 * H(d2) to P1, and both set m' = m + d1 + d2 = x + r_x; then m_z = m' >>_arith t.
 *   xs: sharing of n elements (read); out: sharing of n elements (written, not xs);
 *   pq: 12 n words (written): <p>, <q> of the pairs, for mpc_verify_trunc.
 * Workspace: MPC_OP_TRUNC.  Waits for the hash check; MPC_ERR_ABORT when a received d disagrees
 * with P0's hash.  The pairs stay pending until mpc_verify_trunc(trunc_call_id = call_id). */
int mpc_trunc(mpc_ctx* ctx, uint64_t call_id, const uint64_t* xs, int64_t n, int t, uint64_t* out,
              uint64_t* pq, void* workspace, size_t workspace_bytes);

/* Pi_BIVerify (Fig. PBDP) of the 2 n inner products of the truncation pairs of
 * mpc_trunc(call_id = trunc_call_id): exactly batch 1 of mpc_verify_matmul, in chunks of at most
 * tuning.trunc_chunk outputs (batches 1, 2, ... of verify_id).  R < 0: the default per chunk.
 * Workspace: MPC_OP_VERIFY_TRUNC (R in R_trunc); trace: mpc_trace_words(MPC_OP_VERIFY_TRUNC, n,
 * 0, 0, t, -1, R) words, chunk after chunk.  Returns as mpc_verify_mult. */
int mpc_verify_trunc(mpc_ctx* ctx, uint64_t verify_id, const uint64_t* pq, int64_t n, int t,
                     uint64_t trunc_call_id, int R, void* workspace, size_t workspace_bytes,
                     uint64_t* trace);

/* H of Pi_Rec on its own (Sec. 2, verifiable reconstruction): the SHA-256 Merkle root (1024-byte
 * leaves of the little-endian byte image, node = SHA-256(left || right), an odd node promoted
 * unchanged, the empty array hashing to SHA-256 of the empty string) of n device words, exactly
 * as mpc_reconstruct computes it for its messages.
 *   data: n device words (borrowed; n >= 0); digest: 32 host bytes (written, FIPS byte order).
 *   Allocates its scratch on the device, synchronises the context's stream and frees it. */
int mpc_hash_u64(mpc_ctx* ctx, const uint64_t* data, int64_t n, uint8_t* digest);

/* Local rearrangement of a sharing (Sec. 2, linear homomorphic property: every party applies the
 * same public map to each component it holds; no communication): out[k] = x[idx[k]], or 0 when
 * idx[k] < 0 (zero padding).  Used for im2col views of convolutions and layout changes.
 *   xs: 6 n_in words; idx: n_out device int64 indices (borrowed); out: 6 n_out words (written).
 *   Indices >= n_in read as 0 (an out-of-range index is never dereferenced). */
int mpc_gather(mpc_ctx* ctx, const uint64_t* xs, int64_t n_in, const int64_t* idx, int64_t n_out,
               uint64_t* out);

/* ---- non-linear layers (Sec. 4.3) -------------------------------------------------------------
 * ReLU(x) = x [x >= 0] and 2x2 max-pool, each one layer with its own verification (reading A14):
 *   - per compare-select stage: edaBits (Fig. edabits: 64 Pi_Mult + one dimension-64 Pi_Inner per
 *     element), Delta = x - r opened with Pi_Rec, msb(x) from a depth-6 parallel-prefix carry
 *     circuit of AND gates (Boolean Pi_Mult over Z_2, 125 per element), B2A of NOT msb with a
 *     daBit (two Pi_Mult), and one Pi_Mult (x - y) [x >= y];
 *   - then Pi_MultVerify of the daBit and final products (batch 0, 3 per element) and
 *     Pi_BIVerify of the edaBit inner products (batch 1) over GR(2^64, 64), Pi_MultVerify of
 *     every AND gate over GF(2^64) = GR(2, 64) (batch 2), and Pi_MultVerify of the edaBit bit
 *     products over GR(2^64, 64) (batch 3, 64 per element; a batch of its own, so that its
 *     vectors keep the form in which only P0's Gram sum is non-zero).
 * Elements are processed in groups padded to n_pad = 64 ceil(n / 64); Boolean values are
 * bit-sliced.  Returns MPC_OK (verified), MPC_ERR_VERIFY, MPC_ERR_ABORT (a Pi_Rec mismatch).
 *   xs: device sharing of n elements (6 n words, read); out: 6 n words (written);
 *   call_id: streams of the layer; verify_id: streams of its verification;
 *   trace (optional, device, zero-filled by the caller): per batch, R + 1 blocks as for
 *     mpc_verify_mult for batches 0 and 1 (R = max(0, ceil(log2 D) - 6), D = products / entries),
 *     then (R2 + 1) blocks of MPC_TRACE_GF_ROUND words for batch 2: zeta', h0 (6), h2 (6) per
 *     round and Delta, then R3 + 1 blocks as for mpc_verify_mult for batch 3. */
#define MPC_TRACE_GF_ROUND 13
int mpc_relu(mpc_ctx* ctx, uint64_t call_id, uint64_t verify_id, const uint64_t* xs, int64_t n,
             uint64_t* out, void* workspace, size_t workspace_bytes, uint64_t* trace);
/* 2x2 / stride-2 max-pool (Sec. 4.3: max(a, b) = b + (a - b)[a >= b], reading N6) of a
 * (B, C, H, W) tensor, H and W even; out has B C (H/2) (W/2) elements.  Stage 0 compares the
 * window pairs ([2i][2j], [2i][2j+1]) and ([2i+1][2j], [2i+1][2j+1]) in one batch, stage 1 the
 * two winners; the comparisons and their verification are mpc_relu's.  Arguments, trace and
 * return codes as mpc_relu. */
int mpc_maxpool2(mpc_ctx* ctx, uint64_t call_id, uint64_t verify_id, const uint64_t* xs, int64_t B,
                 int64_t C, int64_t H, int64_t W, uint64_t* out, void* workspace,
                 size_t workspace_bytes, uint64_t* trace);

/* Ledger (the communication that Table 1 and Sec. 4.2 count): bytes[phase * MPC_NPROTO + proto]
 * of every message sent so far, and the message count.  Hash messages count 32 bytes. */
int mpc_ledger(const mpc_ctx* ctx, uint64_t* bytes, uint64_t* messages);
void mpc_ledger_reset(mpc_ctx* ctx);

/* Arm a one-shot fault (the actively corrupted party of Sec. 2's security model, whose cheating
 * the checks must catch, with abort): the next message delivered at `site` has element
 * (index mod length) XORed with xor_mask (MPC_SITE_HIGH_BIT ignores xor_mask and uses 2^63).
 * Host side only; it never faults the device. */
int mpc_inject_fault(mpc_ctx* ctx, int site, uint64_t index, uint64_t xor_mask);

/* Phase timers: with profiling on, the library brackets each phase of its work with CUDA events
 * on the context's stream (no synchronisation).  mpc_profile(ctx, 1) clears and starts,
 * mpc_profile(ctx, 0) stops; mpc_profile_read() waits for the stream and returns, per phase, the
 * summed milliseconds and the number of intervals recorded since the last read. */
enum {
  MPC_PROF_SHARE = 0,              /* input sharing                                         */
  MPC_PROF_MULT = 1,               /* Pi_Mult                                               */
  MPC_PROF_TRUNC_PAIRS = 2,        /* Pi_Trunc preprocessing (trunc pairs and their messages) */
  MPC_PROF_GEMM = 3,               /* the local products of Pi_Inner (one interval / party) */
  MPC_PROF_EXCHANGE = 4,           /* Gamma and m_Z messages, reconstruction of m_Z, m >> t  */
  MPC_PROF_VERIFY_GEMM = 5,        /* batch 0 of Pi_BIVerify (folds, rounds, InnerVerify)   */
  MPC_PROF_TRUNC_SETUP = 6,        /* batch 1: challenge, bits, powers r^(2e), z            */
  MPC_PROF_TRUNC_S = 7,            /* batch 1: S_{j,j'} = sum_e r^(2e) b1_j b2_j'           */
  MPC_PROF_TRUNC_ROUNDS = 8,       /* batch 1: the rounds that fold the 64 bits per output  */
  MPC_PROF_TRUNC_MATERIALIZE = 9,  /* batch 1: folded vectors of the remaining rounds       */
  MPC_PROF_TRUNC_TAIL = 10,        /* batch 1: remaining rounds and Pi_InnerVerify          */
  MPC_PROF_REC = 11,               /* Pi_Rec of outputs                                     */
  MPC_PROF_VERIFY_MULT = 12,       /* Pi_MultVerify                                         */
  /* kernel-level intervals, nested inside the phases above (not added to them):           */
  MPC_PROF_K_LIMB_GEMM = 13,       /* the tensor-core kernel of each limb-split product     */
  MPC_PROF_K_TRUNC_S = 14,         /* the tensor-core kernel of the trunc-batch S matrix     */
  MPC_PROF_K_GR_MATMUL = 15,       /* tensor-core GR-matrix products (folds, tables)        */
  MPC_PROF_K_GRAM = 16,            /* tensor-core Gram sums of the dense rounds              */
  MPC_PROF_K_GR_MUL_ROWS = 17,     /* elementwise GR products (CUDA cores)                   */
  MPC_PROF_NONLINEAR = 18,         /* a non-linear layer (ReLU / max-pool), its verification */
  MPC_NPROF = 19
};
int mpc_profile(mpc_ctx* ctx, int enable);
/* work (may be NULL): per interval id, the algorithmic u64 multiply-accumulates of the kernels
 * timed under that id (M N K per limb-split product, 4096 per bit pair, coefficient and output
 * of the S matrix, R 64 64 per GR-matrix product, 4 Dh 4096 per Gram call, 4096 per elementwise
 * GR product); 0 for the phases. */
int mpc_profile_read(mpc_ctx* ctx, double* ms /* MPC_NPROF */, uint64_t* count /* MPC_NPROF */,
                     double* work /* MPC_NPROF */);

/* Test hook for failure detection (no counterpart in the paper): one thread waits, with the
 * bounded-wait helper of the tensor-core kernels and a limit of `cycles` (1 .. 1e8) clock cycles,
 * on an mbarrier that nothing arrives at.  The wait runs out, the kernel records the expiry in
 * the context's status word and returns, and the call reports it as any expired wait is
 * reported: MPC_ERR_TIMEOUT, with the context aborted (every later call returns
 * MPC_ERR_ABORT).  The device stays usable.  For tests only. */
int mpc_test_wait_expires(mpc_ctx* ctx, int64_t cycles);

/* Number of kernel launches the library has issued in this process (all contexts). */
uint64_t mpc_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* MPC3_H */
