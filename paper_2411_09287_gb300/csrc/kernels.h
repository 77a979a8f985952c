// Host-side launchers of libmpc3's kernels (internal interface between the protocol code in
// api.cu and the kernels).  Every launcher enqueues on `st` and returns nothing; launch errors
// are collected by the protocol code with cudaGetLastError().
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mpc3 {

// ---- u64 GEMM on CUDA cores ----------------------------------------------------------------
// An operand is value(r, c) = scale * (p0[r, c] + s1 * p1[r, c]) with element (r, c) stored at
// p[r*ld + c] (trans = 0) or p[c*ld + r] (trans = 1); p1 may be null.
struct Opnd {
  const u64* p0;
  const u64* p1;
  long long ld;
  u64 s1;
  u64 scale;
  int trans;
};
struct GemmTerm {
  Opnd A;   // M x K
  Opnd B;   // K x N
};
// out[i] = acc_sign*acc + add0[i] + add1[i] + prf_sign*PRF(key, tag, obj, i), i = r*ldc + c,
// or, with atomic = 1, out[r*ldc + c] += acc_sign*acc (split-K accumulation).
struct Epi {
  int atomic;
  u64 acc_sign;
  const u64* add0;
  long long ld_add0;   // row stride of add0 (0: same index as out)
  const u64* add1;
  u64 prf_sign;
  Key key;
  u32 tag;
  u64 obj;
  u64* out;
  long long ldc;
};
// Up to GRAM_BATCH_MAX independent 64 x 64 Gram sums out_i += sign_i sum_k A_i[:, k] B_i[k, :]
// (each a one-term product, K deep, with an atomic epilogue) in one launch.
constexpr int GRAM_BATCH_MAX = 8;
void gemm_u64_gram_batch(cudaStream_t st, long long K, int n, const GemmTerm* terms,
                         const Epi* epis, int nsplit);
// C(M x N) = sum over terms of A_t (M x K) * B_t (K x N), then the epilogue.  nsplit > 1 splits
// K across grid.z and requires epi.atomic = 1.
void gemm_u64(cudaStream_t st, long long M, long long N, long long K, int nterms,
              const GemmTerm* terms, const Epi& epi, int nsplit);
// The same product in 16 x 16 output tiles, one output per thread and no split: for small
// products (a few thousand outputs, short K) that one 64 x 64 tile would leave on one SM.
void gemm_u64_small(cudaStream_t st, long long M, long long N, long long K, int nterms,
                    const GemmTerm* terms, const Epi& epi);

// ---- exact u64 GEMM on the tcgen05 tensor cores (limb_gemm_tc.cu) ---------------------------
// Same contract as gemm_u64 without split-K (epi.atomic must be 0; returns -1 otherwise, -2 if
// the tensor maps cannot be encoded).  scratch: limb_tc_scratch_bytes(M, N, K, nterms) bytes,
// 256-byte aligned (the bf16 digit planes of both operands).  A bounded wait that expires
// sets err_flag in *err and leaves the output undefined.
size_t limb_tc_scratch_bytes(long long M, long long N, long long K, int nterms);
// ev0 / ev1 (may be null) are recorded on st around the tensor-core kernel alone.
int limb_gemm_tc(cudaStream_t st, long long M, long long N, long long K, int nterms,
                 const GemmTerm* terms, const Epi& epi, void* scratch, unsigned* err,
                 unsigned err_flag, cudaEvent_t ev0, cudaEvent_t ev1, int split_min = 0);

// Row map of a GR matrix product: logical row rho sits at word offset (rho % q) s1 + (rho / q) s2
// (q = 0: rho s1).  q must be a multiple of 128.
struct GrRowMap {
  long long q, s1, s2;
};
// GR-matrix product on the tensor cores, exact: out[rho][c] = add0[rho][c] +
// sum_k A[rho][k] M[k][c] (k, c < 64, M row-major 64 x 64) for rows rho < R.  A row rho at
// p0 + in(rho) (minus p1 + in(rho): s1 must be -1 when p1 is given; returns -1 otherwise), or
// with a_bits the bits of the word p0[in(rho)]; matrix rho / mrows at Mmat + 4096 (rho / mrows)
// (mrows = 0: one matrix, else a multiple of 128); out row rho at out + om(rho), written only
// when om(rho) < out_lim (0: no limit); add0 (may be null) row rho at add0 + rho ld_add0
// (0: 64).  Needs 16-byte aligned bases and even row strides (returns -1 otherwise).
struct GrMMArgs {
  long long R;
  const u64* p0;
  const u64* p1;
  u64 s1;
  GrRowMap in;
  int a_bits;
  const u64* Mmat;
  long long mrows;
  const u64* add0;
  long long ld_add0;
  u64* out;
  GrRowMap om;
  long long out_lim;
  long long qvalid;   // > 0: only rows with rho % in.q < qvalid exist (padded segments)
  int add0_in;        // add0 row rho at add0 + in(rho) (the input map) instead of rho ld_add0
  int tma;            // 1: the A rows of the plain and fold modes are loaded by TMA; 2: and the
                      // A operand sits in tensor memory
  int drain_warps;    // 8 (default) or 16 drain warps
  int out_tma;        // set by the launcher: bit-operand tiles leave by TMA stores (tensor map of
                      // out and om in place of p1's)
};
int gr_matmul_tc_ex(cudaStream_t st, const GrMMArgs& a, unsigned* err, unsigned err_flag);

// One job of a batched tensor-core Gram launch.  u = a0 + sa1 a1 and v = b0 + sb1 b1 (a1, b1 may
// be null; every pointer 16-byte aligned) are vectors of GR elements (rows of 64 words,
// contiguous); over their Dh element pairs (2i, 2i + 1) the job adds, mod 2^64,
//   P[0] += sign G(u_e, v_e),  P[off_oo] += sign G(u_o, v_o),  P[off_x] += sign (G(u_e, v_o) + G(u_o, v_e))
// with G(u, v)[a][b] = sum_i u_i[a] v_i[b] a 64 x 64 block.
struct GramJob {
  const u64* a0;
  const u64* a1;
  u64 sa1;
  const u64* b0;
  const u64* b1;
  u64 sb1;
  u64* P;
  u64 sign;
};
constexpr int GRAM_JOBS_MAX = 8;
struct GramJobs {
  GramJob j[GRAM_JOBS_MAX];
  int n;
  long long off_oo, off_x;   // word offsets of the odd-odd and cross blocks from a job's P
};
// Every job of `jobs`: one launch for the single-source jobs and one for those with a second
// source (nsplit: CTAs per parity shared by a launch's jobs, 0 = half the SMs).  Returns -1 for a
// bad job (null or misaligned pointers), 0 otherwise.
int gram_jobs_tc(cudaStream_t st, long long Dh, const GramJobs& jobs, unsigned* err,
                 unsigned err_flag, int nsplit = 0);
// P[0..2] (3 x 4096 words, accumulated mod 2^64) += the Gram sums G(x_e, y_e), G(x_o, y_o),
// G(x_e, y_o) + G(x_o, y_e) over the Dh element pairs (x_{2i}, x_{2i+1}) of x and y (rows of 64
// words, contiguous).  Exact, on the tensor cores; returns -1 for misaligned inputs.
int gram3_tc(cudaStream_t st, long long Dh, const u64* x, const u64* y, u64* P, unsigned* err,
             unsigned err_flag, int nsplit = 0);

// ---- elementwise protocol kernels (prf_kernels.cu) ------------------------------------------
void launch_share_input(cudaStream_t st, const u64* x, long long n, Key k01, Key k02, u64 obj,
                        u64* s6, u64* p0_out_m);
void launch_fill_masks(cudaStream_t st, long long n, Key k01, Key k02, u32 purpose, u64 obj,
                       u64* s6);
void launch_mult_offline(cudaStream_t st, const u64* xs, const u64* ys, long long n, Key k01,
                         Key k02, u64 obj, u64* zs, u64* p0_out_g2);
void launch_mult_online(cudaStream_t st, const u64* xs, const u64* ys, long long n, Key k01,
                        u64 obj, const u64* p2_in_g2, u64* p1_out, u64* p2_out);
// m = own + received for P1 and P2; with t >= 0 also writes the truncated m (>>_arith t) into
// out_s6 (P1.m, P2.m components) when out_s6 != null.
void launch_exchange_finish(cudaStream_t st, long long n, const u64* p1_own, const u64* p1_in,
                            const u64* p2_own, const u64* p2_in, u64* zs, int t, u64* outs);
// row_keys (device, one object id per output row of N outputs, or null): the truncation bits of
// output e come from the streams of object row_keys[e / N] at word e mod N
void launch_trunc_p0(cudaStream_t st, long long E, Key k01, Key k02, u64 obj, int t, u64* zpre,
                     u64* zout, u64* pq, u64* p0_out_gp2, u64* p0_out_gq2, u64* p1_out_mp,
                     u64* p1_out_mq, const u64* row_keys, long long N);
void launch_trunc_finish(cudaStream_t st, long long E, Key k01, Key k02, u64 obj, int t,
                         const u64* p1_in_mp, const u64* p1_in_mq, const u64* p2_in_mp,
                         const u64* p2_in_mq, const u64* p2_gp2, const u64* p2_gq2,
                         const u64* p1_mp1, const u64* p1_mq1, u64* zpre, u64* zout, u64* pq,
                         const u64* row_keys, long long N);
void launch_xor_one(cudaStream_t st, u64* p, u64 mask);
void launch_open_p1(cudaStream_t st, const u64* p1_m, const u64* p1_r1, const u64* p1_in_r2,
                    long long n, u64* out);

// ---- SHA-256 Merkle hash (sha_kernels.cu) ---------------------------------------------------
// Merkle hash of Pi_Rec: 1024-byte leaves, subtree roots of 64 aligned leaves per CTA.
constexpr long long HASH_LEAF_BYTES = 1024;
constexpr long long HASH_CTA_LEAVES = 64;
constexpr long long hash_scratch_words_for(long long n) {
  return 16 * (((8 * n + HASH_LEAF_BYTES - 1) / HASH_LEAF_BYTES > 1
                    ? (8 * n + HASH_LEAF_BYTES - 1) / HASH_LEAF_BYTES
                    : 1) +
               HASH_CTA_LEAVES - 1) /
         HASH_CTA_LEAVES;
}
// digest (8 words) of the n-word array; scratch needs hash_scratch_words(n) 32-bit words.
void launch_hash_u64(cudaStream_t st, const u64* data, long long n, u32* scratch, u32* digest);
void launch_digest_check(cudaStream_t st, const u32* a0, const u32* b0, const u32* a1,
                         const u32* b1, const u32* a2, const u32* b2, u32* status, u32 flag);
size_t hash_scratch_words(long long n);

// ---- GR(2^64, 64) kernels (gr_kernels.cu) ---------------------------------------------------
void launch_gr_random_shared(cudaStream_t st, long long n, Key k01, Key k02, Key k12,
                             u32 purpose, u64 obj, u64* s6);
void launch_gr_powers(cudaStream_t st, const u64* a, long long n, u64* table);
void launch_gr_mul1(cudaStream_t st, const u64* a, const u64* b, u64* out);
void launch_gr_lincomb(cudaStream_t st, const u64* ca, const u64* a, const u64* cb, const u64* b,
                       u64* out);
void launch_gr_mulmat2(cudaStream_t st, const u64* a, const u64* b, u64* M);
void launch_gr_inverses(cudaStream_t st, u64* out);
void launch_gr_lagrange(cudaStream_t st, const u64* zeta_prime, int mode, const u64* inv,
                        u64* coef);
void launch_gr_fold_reduce(cudaStream_t st, const u64* P, int n, u64* out);
void launch_gr_combine_z(cudaStream_t st, const u64* coef, const u64* h0, const u64* h2,
                         const u64* z, u64* znew);
void launch_gr_scale_rows(cudaStream_t st, const u64* pw, const u64* s, long long n, u64* out);
void launch_gr_lift(cudaStream_t st, const u64* s, long long n, u64* out);
// First-round party sums and folds of a claim whose y vectors are lifted ring words (one word per
// element, components null when absent): S (12 x 64 words, accumulated) receives the party sums
// of the even pairs at S[0..2], of the cross terms at S[3..5] and of the odd pairs at S[9..11];
// out_i = lift(Y_{2i}) + f (Y_{2i+1} - Y_{2i}).  Words at or past D read as 0.
void launch_gram_lifted(cudaStream_t st, const u64* const x[6], const u64* const y[6], long long Dh,
                        long long D, u64* S);
void launch_fold_lifted(cudaStream_t st, const u64* Y, long long Dh, long long D, const u64* f,
                        u64* out);
void launch_neg_copy(cudaStream_t st, const u64* a, long long n, u64* out);
void launch_gr_check_zero(cudaStream_t st, const u64* v, u32* status, u32 flag);
void launch_trunc_u(cudaStream_t st, const u64* r, int t, u64* u);
void launch_trunc_round_h(cudaStream_t st, const u64* V, const u64* W, const u64* S, int k,
                          const u64* lam, u64* out);
void launch_trunc_update_vw(cudaStream_t st, u64* V, u64* W, int k, const u64* coef);
// out[c] += sum_{e < n} A[c * lda + e] * R[e] (R: n GR elements), c < nrows <= 16, atomically
void launch_scalar_gr_sum(cudaStream_t st, long long n, const u64* A, long long lda, int nrows,
                          const u64* R, u64* out);
// out[e] = a[e] * b[e] (GR products of n row pairs; out may alias a or b)
void launch_gr_mul_rows(cudaStream_t st, long long n, const u64* a, const u64* b, u64* out);
// out[i] = src[idx(i)] (rows of 64 words), idx(i) = ((i mul) / div) mod m (m = 0: no mod).
void launch_gather_rows_affine(cudaStream_t st, long long n, const u64* src, long long mul,
                               long long div, long long m, u64* out);
// out[c] = sum over h < nper of in[c nper + h] (rows of 64 words), c < ncomp.
void launch_block_rowsum(cudaStream_t st, int ncomp, long long nper, const u64* in, u64* out);
// M + 4096 i = multiplication matrix (M[b][c] = coefficient c of g x^b) of g = src + i stride,
// i < n.
void launch_gr_mulmat_batch(cudaStream_t st, long long n, const u64* src, long long stride,
                            u64* M);
// out (cols x rows) = transpose of in viewed as rows x cols; source indices >= n read as 0.
void launch_word_transpose(cudaStream_t st, long long rows, long long cols, long long n,
                           const u64* in, u64* out);
void launch_trunc_materialize(cudaStream_t st, long long E, const u64* words, const u64* VW,
                              const u64* R, int kd, u64* out);
void launch_gr_rec1(cudaStream_t st, const u64* s6, u64 xor_mask, int xor_idx, u64* out,
                    u32* status, u32 flag);
void launch_gr_inner_finish_all(cudaStream_t st, const u64* S, Key k01, Key k02, u32 purpose,
                                u64 obj, u64* h6);
void launch_gr_quad_combine(cudaStream_t st, const u64* lam, const u64* S00, const u64* S01,
                            const u64* S10, const u64* S11, u64* out);
void launch_mode_consts(cudaStream_t st, int mode, u64* cst);
// PRF words off .. off + n - 1 of one stream into out[0 .. n) (e.g. the truncation bits b1, b2
// of the outputs of one verification chunk)
void launch_prf_words(cudaStream_t st, long long n, Key key, u32 tag, u64 obj, u64* out,
                      long long off = 0);
// the same for a row-keyed truncation-bit stream: word e = word e mod N of object row_keys[e / N]
void launch_prf_words_keyed(cudaStream_t st, long long n, Key key, u32 tag, const u64* row_keys,
                            long long N, u64* out, long long off);

// ---- trunc-batch S matrix on the tensor cores (trunc_s.cu) ----------------------------------
void launch_trunc_limb_table(cudaStream_t st, const u64* Tlo, long long L, unsigned char* TL8);
// BT[j][w] = bit j of words[64 w + i] at bit i, for w < Epad / 64
void launch_trunc_bit_transpose(cudaStream_t st, const u64* words, long long Epad, u64* BT);
// S_hi[e_hi][64 j + j'][coeff] for e_hi < nhi; returns -2 if the tensor map cannot be encoded.
// A bounded wait that expires sets err_flag in *err (the output is then undefined).
int launch_trunc_s_tc(cudaStream_t st, const u64* B1T, const u64* B2T, long long Epad,
                      const unsigned char* TL8, long long L, long long nhi, u64* S_hi,
                      unsigned* err, unsigned err_flag);
void launch_fold_reduce_strided(cudaStream_t st, const u64* P, long long ld, int npairs, u64* out);

// ---- non-linear layers: Boolean sharings, AND gates, GF(2^64) (nonlinear.cu) ------------------
void launch_and_offline(cudaStream_t st, const u64* xs, const u64* ys, long long nw, Key k01, Key k02,
                        u32 purpose, u64 obj, u64* zs, u64* g2_out);
void launch_and_online(cudaStream_t st, const u64* xs, const u64* ys, long long nw, Key k01,
                       u32 purpose, u64 obj, const u64* g2_in, u64* p1_out, u64* p2_out);
void launch_xor_finish(cudaStream_t st, long long nw, const u64* p1_own, const u64* p1_in,
                       const u64* p2_own, const u64* p2_in, u64* zs);
void launch_bits_to_arith(cudaStream_t st, const u64* bits, long long n, int kind, u64* out);
void launch_lin_apb_m2c(cudaStream_t st, long long n, const u64* a, const u64* b, const u64* c, u64* out);
void launch_eda_inner_offline(cudaStream_t st, long long np, Key k01, Key k02, u64 obj, u64* zs,
                              u64* g2_out);
void launch_eda_inner_online(cudaStream_t st, const u64* mbits, const u64* rp, long long np, Key k01,
                             u64 obj, const u64* g2_in, u64* p1_out, u64* p2_out);
void launch_eda_compose(cudaStream_t st, const u64* mbits, const u64* rp, const u64* z, long long np,
                        u64* ra);
void launch_msb_leaves(cudaStream_t st, const u64* rbits, const u64* dplanes, long long W, u64* G,
                       u64* P);
void launch_msb_gather(cudaStream_t st, const u64* G, const u64* P, int C, int root, long long W,
                       u64* X, u64* Y);
void launch_msb_combine(cudaStream_t st, const u64* G, const u64* Z, int C, int root, long long W,
                        u64* Gout, u64* Pout);
void launch_msb_out(cudaStream_t st, const u64* rbits, const u64* Groot, const u64* d63, long long W,
                    int negate, u64* out);
void launch_bxor(cudaStream_t st, long long n6, const u64* a, const u64* b, u64* out);
void launch_b2a_apply(cudaStream_t st, const u64* dbits, const u64* ra, long long n, u64* out);
void launch_addsub(cudaStream_t st, long long n, const u64* a, const u64* b, int sub, u64* out);
void launch_open_xor(cudaStream_t st, const u64* m, const u64* r1, const u64* r2_in, long long n,
                     u64* out);
// First round of the edaBit inner-product batch from the bits (see nonlinear.cu): per-element
// party-sum words (6 rows of ld words) and the x fold (A: r^g f per element g).
void launch_eda_r1_sums(cudaStream_t st, const u64* mbits, const u64* rp, long long np, long long e0,
                        long long ld, u64* out);
void launch_eda_x_fold(cudaStream_t st, const u64* mbits, long long np, long long e0, const u64* pw,
                       const u64* A, u64* x2, u64* x4);
void launch_eda_tran(cudaStream_t st, const u64* mbits, const u64* rp, long long np, const u64* pw,
                     long long e0, u64* x2, u64* x4, u64* const* y_dev);
void launch_gf_powers(cudaStream_t st, const u64* r, long long n, u64* out);
void launch_gf_tran(cudaStream_t st, const u64* X, const u64* Y, const u64* Z, long long nw,
                    const u64* pw, long long ld, u64* xo, u64* yo, u64* zsum);
void launch_gf_party_sums(cudaStream_t st, const u64* const u[6], const u64* const v[6], long long D,
                          long long stride, long long off, int fold, u64 fa, u64 fb, u64* S);
// The GF fold of the six components of x and of y (component c at c * cap in, c * ocap out).
void launch_gf_fold6x2(cudaStream_t st, const u64* xv, const u64* yv, long long cap, long long D,
                       const u64* zeta, u64* xo, u64* yo, long long ocap);
void launch_gf_inner_finish(cudaStream_t st, const u64* S, Key k01, Key k02, u32 purpose, u64 obj,
                            u64* h6);
void launch_gf_random_shared(cudaStream_t st, Key k01, Key k02, Key k12, u32 purpose, u64 obj,
                             u64* s6);
void launch_gf_rec1(cudaStream_t st, const u64* s6, u64 xor_mask, u64* out, u32* status, u32 flag);
void launch_gf_lagrange(cudaStream_t st, const u64* zeta, u64* coef);
void launch_gf_combine_z(cudaStream_t st, const u64* coef, const u64* h0, const u64* h2, const u64* z,
                         u64* zo);
void launch_gf_mult_alpha(cudaStream_t st, const u64* const x[6], const u64* a6, long long D,
                          long long ld, Key k01, Key k02, u64 obj, u64* xa);
void launch_gather(cudaStream_t st, const u64* xs, long long n_in, const long long* idx,
                   long long n_out, u64* out);
void launch_window_gather(cudaStream_t st, const u64* x, long long BC, long long H, long long W,
                          long long np, u64* left, u64* right);
void launch_gf_check_zero(cudaStream_t st, const u64* d, u32* status, u32 flag);
// arithmetic Pi_Mult with the streams of `purpose` (prf_kernels.cu)
void launch_mult_offline_p(cudaStream_t st, const u64* xs, const u64* ys, long long n, Key k01,
                           Key k02, u32 purpose, u64 obj, u64* zs, u64* p0_out_g2);
void launch_mult_online_p(cudaStream_t st, const u64* xs, const u64* ys, long long n, Key k01,
                          u32 purpose, u64 obj, const u64* p2_in_g2, u64* p1_out, u64* p2_out);

// ---- layer-level calls (layer_kernels.cu) ----------------------------------------------------
// Geometry of a convolution: NCHW input (B, C, H, W), kh x kw kernel, stride, zero padding; the
// output is Ho x Wo per image.
struct ConvGeom {
  long long B, C, H, W, kh, kw, stride, pad, Ho, Wo;
};
// out[i] = floor(x[i] 2^k) (saturating, NaN -> 0) / out[i] = (signed) v[i] / 2^k
void launch_encode_fixed(cudaStream_t st, const double* x, long long n, int k, u64* out);
void launch_decode_fixed(cudaStream_t st, const u64* v, long long n, int k, double* out);
// the im2col rows of all six components of x: cols holds 6 (B Ho Wo) (C kh kw) words
void launch_im2col(cudaStream_t st, const u64* x, const ConvGeom& g, u64* cols);
// the mask-switch differences of a standalone truncation and its online shift
void launch_trunc_remask(cudaStream_t st, const u64* xs, const u64* rx, long long n, u64* d1_p1,
                         u64* d2_p2, u64* d1_p0, u64* d2_p0);
void launch_trunc_online(cudaStream_t st, const u64* xs, long long n, const u64* d1,
                         const u64* d2_at_p1, const u64* d1_at_p2, const u64* d2, int t,
                         u64* out);

// test hook: one thread's bounded wait (limit `cycles`) on an mbarrier nothing arrives at
void launch_wait_expires(cudaStream_t st, long long cycles, unsigned* err, unsigned err_flag);

}  // namespace mpc3
