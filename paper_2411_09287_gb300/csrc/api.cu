// libmpc3: the C-ABI and the protocol driver.  Every protocol step runs in the kernels of this
// library; the host code here only sequences them, moves messages between the three simulated
// parties (device-to-device copies counted in the ledger) and carves the caller's workspace.
//
// Paper map: mpc_share_input = Pi_<.>^{l,0} (Sec. 2); mpc_mult = Pi_Mult (Fig. MultP);
// mpc_matmul = Pi_Inner per output (Fig. DPP, Sec. 4.1) + Pi_Trunc (Fig. trunc);
// mpc_verify_mult = Pi_MultVerify (Fig. PPEV); mpc_verify_matmul = Pi_BIVerify (Fig. PBDP);
// both use Pi_Tran (Fig. MTP), Pi_Reduce (Fig. Reduce), Pi_InnerVerify (Fig. DPV);
// mpc_reconstruct = Pi_Rec (Sec. 2).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <set>
#include <string>
#include <vector>

#include "mpc3.h"
#include "kernels.h"

using namespace mpc3;

// ---- kernel launch accounting: every launcher called from this file is counted ----------------
namespace {
unsigned long long g_launches = 0;
template <class F, class... A>
inline void counted(int k, F f, A... a) {
  g_launches += (unsigned long long)k;
  f(a...);
}
}  // namespace
#define gemm_u64(...) counted(1, mpc3::gemm_u64, __VA_ARGS__)
#define gemm_u64_small(...) counted(1, mpc3::gemm_u64_small, __VA_ARGS__)
#define launch_share_input(...) counted(1, mpc3::launch_share_input, __VA_ARGS__)
#define launch_fill_masks(...) counted(1, mpc3::launch_fill_masks, __VA_ARGS__)
#define launch_mult_offline(...) counted(1, mpc3::launch_mult_offline, __VA_ARGS__)
#define launch_mult_online(...) counted(1, mpc3::launch_mult_online, __VA_ARGS__)
#define launch_exchange_finish(...) counted(1, mpc3::launch_exchange_finish, __VA_ARGS__)
#define launch_trunc_p0(...) counted(1, mpc3::launch_trunc_p0, __VA_ARGS__)
#define launch_trunc_finish(...) counted(1, mpc3::launch_trunc_finish, __VA_ARGS__)
#define launch_xor_one(...) counted(1, mpc3::launch_xor_one, __VA_ARGS__)
#define launch_open_p1(...) counted(1, mpc3::launch_open_p1, __VA_ARGS__)
#define launch_hash_u64(...) counted(2, mpc3::launch_hash_u64, __VA_ARGS__)
#define launch_digest_check(...) counted(1, mpc3::launch_digest_check, __VA_ARGS__)
#define launch_gr_random_shared(...) counted(1, mpc3::launch_gr_random_shared, __VA_ARGS__)
#define launch_gr_powers(...) counted(1, mpc3::launch_gr_powers, __VA_ARGS__)
#define launch_gr_mul1(...) counted(1, mpc3::launch_gr_mul1, __VA_ARGS__)
#define launch_gr_lincomb(...) counted(1, mpc3::launch_gr_lincomb, __VA_ARGS__)
#define launch_gr_mulmat2(...) counted(1, mpc3::launch_gr_mulmat2, __VA_ARGS__)
#define launch_gr_inverses(...) counted(1, mpc3::launch_gr_inverses, __VA_ARGS__)
#define launch_gr_lagrange(...) counted(1, mpc3::launch_gr_lagrange, __VA_ARGS__)
#define launch_gr_fold_reduce(...) counted(1, mpc3::launch_gr_fold_reduce, __VA_ARGS__)
#define launch_gr_combine_z(...) counted(1, mpc3::launch_gr_combine_z, __VA_ARGS__)
#define launch_gr_scale_rows(...) counted(1, mpc3::launch_gr_scale_rows, __VA_ARGS__)
#define launch_gr_lift(...) counted(1, mpc3::launch_gr_lift, __VA_ARGS__)
#define launch_gram_lifted(...) counted(1, mpc3::launch_gram_lifted, __VA_ARGS__)
#define launch_fold_lifted(...) counted(1, mpc3::launch_fold_lifted, __VA_ARGS__)
#define launch_neg_copy(...) counted(1, mpc3::launch_neg_copy, __VA_ARGS__)
#define launch_gr_check_zero(...) counted(1, mpc3::launch_gr_check_zero, __VA_ARGS__)
#define launch_trunc_u(...) counted(1, mpc3::launch_trunc_u, __VA_ARGS__)
#define launch_trunc_round_h(...) counted(1, mpc3::launch_trunc_round_h, __VA_ARGS__)
#define launch_trunc_update_vw(...) counted(1, mpc3::launch_trunc_update_vw, __VA_ARGS__)
#define launch_trunc_materialize(...) counted(1, mpc3::launch_trunc_materialize, __VA_ARGS__)
#define launch_gr_mul_rows(...) counted(1, mpc3::launch_gr_mul_rows, __VA_ARGS__)
#define launch_gather_rows_affine(...) counted(1, mpc3::launch_gather_rows_affine, __VA_ARGS__)
#define launch_block_rowsum(...) counted(1, mpc3::launch_block_rowsum, __VA_ARGS__)
#define launch_gr_mulmat_batch(...) counted(1, mpc3::launch_gr_mulmat_batch, __VA_ARGS__)
#define launch_word_transpose(...) counted(1, mpc3::launch_word_transpose, __VA_ARGS__)
#define launch_scalar_gr_sum(...) counted(1, mpc3::launch_scalar_gr_sum, __VA_ARGS__)
#define launch_gr_rec1(...) counted(1, mpc3::launch_gr_rec1, __VA_ARGS__)
#define launch_gr_inner_finish_all(...) counted(1, mpc3::launch_gr_inner_finish_all, __VA_ARGS__)
#define launch_gr_quad_combine(...) counted(1, mpc3::launch_gr_quad_combine, __VA_ARGS__)
#define launch_mode_consts(...) counted(1, mpc3::launch_mode_consts, __VA_ARGS__)
#define launch_prf_words(...) counted(1, mpc3::launch_prf_words, __VA_ARGS__)
#define launch_prf_words_keyed(...) counted(1, mpc3::launch_prf_words_keyed, __VA_ARGS__)
#define launch_trunc_limb_table(...) counted(1, mpc3::launch_trunc_limb_table, __VA_ARGS__)
#define launch_trunc_bit_transpose(...) counted(1, mpc3::launch_trunc_bit_transpose, __VA_ARGS__)
#define launch_fold_reduce_strided(...) counted(1, mpc3::launch_fold_reduce_strided, __VA_ARGS__)

namespace {

constexpr u32 ST_ABORT = 1u;    // a Pi_Rec check failed
constexpr u32 ST_VERIFY = 2u;   // Delta != 0
constexpr u32 ST_TIMEOUT = 4u;  // a bounded device wait expired

// device constants block (words)
constexpr int CST_INV = 0;      // 192: x^-1, (1-x)^-1, (x(x-1))^-1
constexpr int CST_LAM = 192;    // 128: 1 - p2, p2
constexpr int CST_ONE = 320;    // 64: the element 1
constexpr int CST_MONE = 384;   // 64: the element -1
constexpr int CST_WORDS = 448;

constexpr int TRACE_ROUND = 832;  // words per round in a verification trace

struct Arena {
  char* base;
  size_t cap;
  size_t off = 0;
  bool dry;
  template <class T>
  T* take(long long count) {
    const size_t bytes = ((size_t)std::max<long long>(count, 1) * sizeof(T) + 255) & ~size_t(255);
    T* p = dry ? nullptr : reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
  bool ok() const { return dry || off <= cap; }
};

struct Fault {
  bool armed = false;
  u64 index = 0;
  u64 mask = 0;
};

__global__ void k_derive_keys(Key master, u32* out) {
  // eta_{0,1}, eta_{0,2}, eta_{1,2}: first 32 bytes of ChaCha20(master, counter 0,
  // nonce (0x0059454B, pair, 0)), pair = 1, 2, 3
  const int pair = threadIdx.x + 1;
  if (pair > 3) return;
  u32 o[16];
  chacha_block(master, 0u, 0x0059454Bu, (u32)pair, 0u, o);
  for (int i = 0; i < 8; ++i) out[(pair - 1) * 8 + i] = o[i];
}

__global__ void k_init_consts(int mode, u64* cst) {
  const int t = threadIdx.x;
  cst[CST_ONE + t] = (t == 0) ? 1ull : 0ull;
  cst[CST_MONE + t] = (t == 0) ? ~0ull : 0ull;
}

inline long long ceil_log2(long long v) {
  long long r = 0;
  while ((1ll << r) < v) ++r;
  return r;
}
inline int default_R(long long D) { return D > 1 ? (int)std::max<long long>(0, ceil_log2(D) - 6) : 0; }

}  // namespace

namespace {
mpc_tuning default_tuning() {
  mpc_tuning t;
  t.trunc_block = 65536;
  t.trunc_chunk = 1ll << 24;
  t.row_split = 0;
  t.tc_combine_min = 32;
  t.gemm_split_min = 8;
  t.gram_split = 76;
  t.fold_batch_max = 65536;
  t.gr_producers = 2;
  t.gr_drain_warps = 8;
  return t;
}
}  // namespace

struct mpc_ctx {
  int device = 0;
  mpc_tuning tune = default_tuning();
  cudaStream_t st = nullptr;
  bool own_stream = false;
  Key k01{}, k02{}, k12{};
  int reduce_mode = MPC_REDUCE_POINT_X;
  int gemm_path = MPC_GEMM_U64;
  u64* cst = nullptr;
  u32* status = nullptr;
  u64 ledger[MPC_NPHASE][MPC_NPROTO] = {};
  u64 nmsg = 0;
  Fault fault[MPC_NSITE];
  bool aborted = false;
  std::set<u64> pending;   // (call_id << 1) | kind, kind 0 = mult, 1 = matmul
  std::string err;
  // phase timers (CUDA events on the context's stream), enabled by mpc_profile()
  struct ProfRec {
    int id;
    cudaEvent_t a, b;
    double work;   // algorithmic u64 multiply-accumulates of a kernel interval
  };
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  // asynchronous uploads (mpc_h2d_async): a copy stream and one event per slot
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copy_ev[MPC_H2D_SLOTS] = {};
  cudaEvent_t order_ev = nullptr;   // the context stream's work before a download
};

namespace {

int fail(mpc_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_check(mpc_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, MPC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return MPC_OK;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, MPC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

cudaEvent_t prof_event(mpc_ctx* c) {
  if (c->pool_used == c->pool.size()) {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    c->pool.push_back(e);
  }
  return c->pool[c->pool_used++];
}

// Times the enclosed stream work as phase `id` when profiling is on.
struct Phase {
  mpc_ctx* c;
  int id;
  double work;
  cudaEvent_t a = nullptr;
  Phase(mpc_ctx* c_, int id_, double work_ = 0.0) : c(c_), id(id_), work(work_) {
    if (c->prof) {
      a = prof_event(c);
      cudaEventRecord(a, c->st);
    }
  }
  ~Phase() {
    if (c->prof) {
      cudaEvent_t b = prof_event(c);
      cudaEventRecord(b, c->st);
      c->recs.push_back({id, a, b, work});
    }
  }
};

int guard(mpc_ctx* ctx) {
  if (!ctx) return MPC_ERR_ARG;
  if (ctx->aborted) return fail(ctx, MPC_ERR_ABORT, "context aborted");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, MPC_ERR_CUDA, cudaGetErrorString(e));
  return MPC_OK;
}

bool id_ok(u64 id) { return id < (1ull << 44); }

// ---- messages -----------------------------------------------------------------------------------
void apply_fault(mpc_ctx* ctx, int site, u64* dst, long long n) {
  if (site == MPC_SITE_GAMMA2 && ctx->fault[MPC_SITE_HIGH_BIT].armed) {
    ctx->fault[MPC_SITE_HIGH_BIT].armed = false;
    ctx->fault[MPC_SITE_GAMMA2] = {true, ctx->fault[MPC_SITE_HIGH_BIT].index, 1ull << 63};
  }
  Fault& f = ctx->fault[site];
  if (f.armed && n > 0) {
    launch_xor_one(ctx->st, dst + (f.index % (u64)n), f.mask);
    f.armed = false;
  }
}

int deliver(mpc_ctx* ctx, int phase, int proto, const u64* src, u64* dst, long long n, int site) {
  if (n > 0) CK(cudaMemcpyAsync(dst, src, (size_t)n * 8, cudaMemcpyDeviceToDevice, ctx->st));
  ctx->ledger[phase][proto] += (u64)n * 8;
  ctx->nmsg += 1;
  if (site >= 0) apply_fault(ctx, site, dst, n);
  return MPC_OK;
}

void count_msgs(mpc_ctx* ctx, int phase, int proto, int count, u64 bytes_each) {
  ctx->ledger[phase][proto] += (u64)count * bytes_each;
  ctx->nmsg += (u64)count;
}

int read_status(mpc_ctx* ctx, u32* out) {
  CK(cudaMemcpyAsync(out, ctx->status, sizeof(u32), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (*out & ST_TIMEOUT) {
    ctx->aborted = true;
    return fail(ctx, MPC_ERR_TIMEOUT, "a bounded device wait expired");
  }
  return MPC_OK;
}

// ---- GEMM helpers -------------------------------------------------------------------------------
Opnd op(const u64* p0, long long ld, int trans = 0, const u64* p1 = nullptr, u64 s1 = 1,
        u64 scale = 1) {
  Opnd o;
  o.p0 = p0; o.p1 = p1; o.ld = ld; o.s1 = s1; o.scale = scale; o.trans = trans;
  return o;
}

Epi epi_store(u64* out, long long ldc) {
  Epi e;
  std::memset(&e, 0, sizeof(e));
  e.atomic = 0; e.acc_sign = 1; e.out = out; e.ldc = ldc;
  return e;
}

Epi epi_atomic(u64* out, long long ldc, u64 sign = 1) {
  Epi e = epi_store(out, ldc);
  e.atomic = 1;
  e.acc_sign = sign;
  return e;
}

// split-K factor of the 64 x 64 Gram products: enough CTAs to fill the GPU down to K ~ 2^12
int nsplit_for(long long K) { return (int)std::min<long long>(1024, std::max<long long>(1, K / 32)); }

// out (atomic, 64x64) += sign * sum_i U_i (x) V_i with U = U0 + su U1, V = V0 + sv V1.
void gram(mpc_ctx* ctx, u64* P, const u64* U0, const u64* U1, u64 su, long long ldu, const u64* V0,
          const u64* V1, u64 sv, long long ldv, long long count, u64 sign) {
  u64 us = 1, vs = 1;
  if (!U0) { U0 = U1; U1 = nullptr; us = su; }
  if (!V0) { V0 = V1; V1 = nullptr; vs = sv; }
  if (!U0 || !V0 || count <= 0) return;
  GemmTerm T;
  T.A = op(U0, ldu, 1, U1, su, us);
  T.B = op(V0, ldv, 0, V1, sv, vs);
  gemm_u64(ctx->st, 64, 64, count, 1, &T, epi_atomic(P, 64, sign), nsplit_for(count));
}

// GR-product arguments with this context's choice of producer and drain variant
GrMMArgs grargs(const mpc_ctx* ctx) {
  GrMMArgs g{};
  g.tma = ctx->tune.gr_producers >= 2 ? ctx->tune.gr_producers - 1 : 0;
  g.drain_warps = ctx->tune.gr_drain_warps;
  return g;
}

// out[i] = add0[i] + (p0[i] + s1 p1[i]) . M for i < R (rows of 64 words, M a 64 x 64 GR
// multiplication matrix): the folds of Pi_Reduce and the products by a fixed GR element.  Tensor
// cores on the limb path, the u64 CUDA-core GEMM otherwise.
int gr_matmul(mpc_ctx* ctx, long long R, const u64* p0, const u64* p1, u64 s1, long long lda,
              const u64* Mmat, const u64* add0, long long ld_add0, u64* out, long long ldc) {
  if (R <= 0) return MPC_OK;
  if (ctx->gemm_path == MPC_GEMM_LIMB_TC) {
    g_launches += 1;
    Phase kp(ctx, MPC_PROF_K_GR_MATMUL, (double)R * 4096);
    GrMMArgs g = grargs(ctx);
    g.R = R;
    g.p0 = p0;
    g.p1 = p1;
    g.s1 = s1;
    g.in = GrRowMap{0, lda, 0};
    g.Mmat = Mmat;
    g.add0 = add0;
    g.ld_add0 = ld_add0 ? ld_add0 : ldc;
    g.out = out;
    g.om = GrRowMap{0, ldc, 0};
    if (gr_matmul_tc_ex(ctx->st, g, ctx->status, ST_TIMEOUT) == 0) return MPC_OK;
    g_launches -= 1;   // misaligned view: fall through to the CUDA-core GEMM
  }
  GemmTerm T;
  T.A = p1 ? op(p0, lda, 0, p1, s1) : op(p0, lda);
  T.B = op(Mmat, 64);
  Epi e = epi_store(out, ldc);
  e.add0 = add0;
  e.ld_add0 = add0 ? ld_add0 : 0;
  gemm_u64(ctx->st, R, 64, 64, 1, &T, e, 1);
  return MPC_OK;
}

// C = A B (+ epilogue) for a one-term product that the limb path runs on the tensor cores
// (scratch: limb_tc_scratch_bytes(M, N, K, 1) bytes) and the u64 path on the CUDA cores.
int dense_gemm(mpc_ctx* ctx, long long M, long long N, long long K, const GemmTerm& T,
               const Epi& e, void* scratch) {
  if (scratch && !e.atomic) {
    g_launches += 4;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ctx->prof) {
      e0 = prof_event(ctx);
      e1 = prof_event(ctx);
      ctx->recs.push_back({MPC_PROF_K_LIMB_GEMM, e0, e1, (double)M * N * K});
    }
    if (limb_gemm_tc(ctx->st, M, N, K, 1, &T, e, scratch, ctx->status, ST_TIMEOUT, e0, e1,
                     ctx->tune.gemm_split_min))
      return fail(ctx, MPC_ERR_CUDA, "tensor-core GEMM setup failed");
    return MPC_OK;
  }
  gemm_u64(ctx->st, M, N, K, 1, &T, e, 1);
  return MPC_OK;
}

// A view of a <.>^{l[x]}-shared vector: component pointers (null = identically zero), row stride.
struct View {
  const u64* c[6];
  long long ld;
};

// Party sums of a secure GR inner product sum_i u_i v_i (Sec. 2 inner product over GR):
//   S0 = sum r_u r_v (P0), S1 = -sum (m_u [r_v]_1 + m_v [r_u]_1) (P1),
//   S2 = sum m_u (m_v - [r_v]_2) - m_v [r_u]_2 (P2).  Pmat: 3 x 4096 scratch; S: 3 x 64 out.
// The same Gram sums collected for one batched launch.
struct GramBatch {
  GemmTerm T[GRAM_BATCH_MAX];
  Epi e[GRAM_BATCH_MAX];
  int n = 0;
  void add(u64* P, const u64* U0, const u64* U1, u64 su, long long ldu, const u64* V0,
           const u64* V1, u64 sv, long long ldv, u64 sign) {
    u64 us = 1, vs = 1;
    if (!U0) { U0 = U1; U1 = nullptr; us = su; }
    if (!V0) { V0 = V1; V1 = nullptr; vs = sv; }
    if (!U0 || !V0 || n >= GRAM_BATCH_MAX) return;
    T[n].A = op(U0, ldu, 1, U1, su, us);
    T[n].B = op(V0, ldv, 0, V1, sv, vs);
    e[n] = epi_atomic(P, 64, sign);
    ++n;
  }
};

int party_sums(mpc_ctx* ctx, const View& u, const View& v, long long count, u64* Pmat, u64* S) {
  CK(cudaMemsetAsync(Pmat, 0, 3 * 4096 * 8, ctx->st));
  const u64 M1 = ~0ull;  // -1
  GramBatch gb;
  gb.add(Pmat, u.c[0], u.c[1], 1, u.ld, v.c[0], v.c[1], 1, v.ld, 1);
  gb.add(Pmat + 4096, u.c[2], nullptr, 1, u.ld, v.c[3], nullptr, 1, v.ld, M1);
  gb.add(Pmat + 4096, v.c[2], nullptr, 1, v.ld, u.c[3], nullptr, 1, u.ld, M1);
  gb.add(Pmat + 8192, u.c[4], nullptr, 1, u.ld, v.c[4], v.c[5], M1, v.ld, 1);
  gb.add(Pmat + 8192, v.c[4], nullptr, 1, v.ld, u.c[5], nullptr, 1, u.ld, M1);
  if (count > 0 && gb.n > 0) {
    g_launches += 1;
    gemm_u64_gram_batch(ctx->st, count, gb.n, gb.T, gb.e, nsplit_for(count));
  }
  launch_gr_fold_reduce(ctx->st, Pmat, 3, S);
  return cuda_check(ctx, "party_sums");
}

// Secure GR inner-product finish (P0's Gamma, P1/P2 cross terms, one exchange); 3 messages.
void inner_finish(mpc_ctx* ctx, const u64* S, u32 purpose, u64 obj, u64* h6) {
  launch_gr_inner_finish_all(ctx->st, S, ctx->k01, ctx->k02, purpose, obj, h6);
  count_msgs(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, 3, 512);
}

// Pi_Rec of one shared GR element (3 shares + 3 hashes); an armed REC_MSG fault corrupts the
// P0 -> P1 share, as for any other Pi_Rec.
void rec1(mpc_ctx* ctx, const u64* s6, u64* out) {
  u64 mask = 0;
  int idx = -1;
  Fault& f = ctx->fault[MPC_SITE_REC_MSG];
  if (f.armed) {
    mask = f.mask;
    idx = (int)(f.index % 64);
    f.armed = false;
  }
  launch_gr_rec1(ctx->st, s6, mask, idx, out, ctx->status, ST_ABORT);
  count_msgs(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, 3, 512);
  count_msgs(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, 3, 32);
}

// <v> random GR element, revealed with Pi_Rec.
void reveal(mpc_ctx* ctx, u32 purpose, u64 obj, u64* tmp6, u64* out) {
  launch_gr_random_shared(ctx->st, 1, ctx->k01, ctx->k02, ctx->k12, purpose, obj, tmp6);
  rec1(ctx, tmp6, out);
}

// ---- verification state ---------------------------------------------------------------------
struct Small {   // per-verification small scratch (all device, from the workspace)
  u64* Pmat;     // 4 x 3 x 4096
  u64* S;        // 5 x 192: S00, S01, S10, S11, Sh2
  u64* h0;       // 384
  u64* h2;       // 384
  u64* z[2];     // 384 each
  u64* coef;     // 448
  u64* zp;       // 64
  u64* r;        // 64
  u64* tmp6;     // 384
  u64* MM;       // 128 x 64
  u64* MA;       // 5 x 4096 (multiplication matrices of alpha components)
  u64* alpha;    // 384
  u64* aux;      // 4 x 64
  u64* Sfull;    // 192
  u64* zinit;    // 384: the claim entering the first round (never round scratch)
};

Small plan_small(Arena& a) {
  Small s;
  s.Pmat = a.take<u64>(4 * 3 * 4096);
  s.S = a.take<u64>(5 * 192);
  s.h0 = a.take<u64>(384);
  s.h2 = a.take<u64>(384);
  s.z[0] = a.take<u64>(384);
  s.z[1] = a.take<u64>(384);
  s.coef = a.take<u64>(448);
  s.zp = a.take<u64>(64);
  s.r = a.take<u64>(64);
  s.tmp6 = a.take<u64>(384);
  s.MM = a.take<u64>(128 * 64);
  s.MA = a.take<u64>(5 * 4096);
  s.alpha = a.take<u64>(384);
  s.aux = a.take<u64>(4 * 64);
  s.Sfull = a.take<u64>(192);
  s.zinit = a.take<u64>(384);
  return s;
}

// A dense claim: x, y vectors of D GR elements (components may be null), claimed z (6 x 64).
struct Vec {
  u64* c[6];
};

struct Dense {
  Vec x[2], y[2];     // ping-pong buffers, capacity cap0 (index 0) and cap1 (index 1)
  long long cap[2];
  int cur = 0;
};

// Inner-verify buffers for a final dimension D.
struct IVBuf {
  u64* xp;    // 6 x (D+1) x 64
  u64* yy;    // 6 x (D+1) x 64
  u64* g2o;   // (D+1) x 64
  u64* g2i;
  u64* p1o;
  u64* p2o;
  u64* p1i;
  u64* p2i;
  u64* zero;  // D x 64 zeros
  u64* delta; // 64
};

IVBuf plan_iv(Arena& a, long long D) {
  IVBuf b;
  const long long w = (D + 1) * 64;
  b.xp = a.take<u64>(6 * w);
  b.yy = a.take<u64>(6 * w);
  b.g2o = a.take<u64>(w);
  b.g2i = a.take<u64>(w);
  b.p1o = a.take<u64>(w);
  b.p2o = a.take<u64>(w);
  b.p1i = a.take<u64>(w);
  b.p2i = a.take<u64>(w);
  b.zero = a.take<u64>(w);
  b.delta = a.take<u64>(64);
  return b;
}

void trace_round(mpc_ctx* ctx, u64* trace, int k, const Small& s) {
  if (!trace) return;
  u64* t = trace + (long long)(k - 1) * TRACE_ROUND;
  cudaMemcpyAsync(t, s.zp, 64 * 8, cudaMemcpyDeviceToDevice, ctx->st);
  cudaMemcpyAsync(t + 64, s.h0, 384 * 8, cudaMemcpyDeviceToDevice, ctx->st);
  cudaMemcpyAsync(t + 448, s.h2, 384 * 8, cudaMemcpyDeviceToDevice, ctx->st);
}

// The part of a Pi_Reduce round after its party sums (in s.S: S00, S01 + S10 (with S10), S11):
// h(0) and h(p2) by secure GR inner products, zeta revealed, the Lagrange weights, the next claim
// zo, and M_zeta (s.MM) for the folds; the fold element is s.coef[0..63].
void round_tail(mpc_ctx* ctx, u64 vid, u32 batch, int k, const u64* z, u64* zo, const Small& s) {
  cudaStream_t st = ctx->st;
  launch_gr_quad_combine(st, ctx->cst + CST_LAM, s.S, s.S + 192, s.S + 384, s.S + 576, s.S + 768);
  const u64 obj = make_obj(vid, batch, (u32)k);
  inner_finish(ctx, s.S, P_VER_H0, obj, s.h0);
  inner_finish(ctx, s.S + 768, P_VER_H2, obj, s.h2);
  reveal(ctx, P_VER_ZETA, obj, s.tmp6, s.zp);
  launch_gr_lagrange(st, s.zp, ctx->reduce_mode, ctx->cst + CST_INV, s.coef);
  launch_gr_combine_z(st, s.coef, s.h0, s.h2, z, zo);
  launch_gr_mulmat2(st, s.coef, nullptr, s.MM);   // M_zeta
}

// One Pi_Reduce round on a dense claim (Fig. Reduce).  x, y: current vectors (D elements, with
// capacity for D+1), z: current claim; writes the folded vectors into xo, yo and z into zo.
// ys (optional): the y vectors are lifted ring words, one word per element (Fig. MTP's y side
// before any fold); y is then not read, the party sums are scalar-weighted row sums and the y
// folds scalar times GR element.
int reduce_round_dense(mpc_ctx* ctx, u64 vid, u32 batch, int k, const Vec& x, const Vec& y,
                       long long D, const u64* z, Vec& xo, Vec& yo, u64* zo, const Small& s,
                       u64* trace, const Vec* ys = nullptr) {
  cudaStream_t st = ctx->st;
  const long long Dh = (D + 1) / 2;
  if (D & 1) {
    for (int c = 0; c < 6; ++c) {
      if (x.c[c]) CK(cudaMemsetAsync(x.c[c] + D * 64, 0, 512, st));
      if (y.c[c] && !ys) CK(cudaMemsetAsync(y.c[c] + D * 64, 0, 512, st));
    }
  }
  View f[2], g[2];
  for (int a = 0; a < 2; ++a) {
    for (int c = 0; c < 6; ++c) {
      f[a].c[c] = x.c[c] ? x.c[c] + 64 * a : nullptr;
      g[a].c[c] = y.c[c] ? y.c[c] + 64 * a : nullptr;
    }
    f[a].ld = 128;
    g[a].ld = 128;
  }
  u64* S00 = s.S;
  u64* S01 = s.S + 192;
  u64* S10 = s.S + 384;
  u64* S11 = s.S + 576;
  int rc;
  // Shape of the truncation batch's dense rounds: x holds only [r]_1 (P0, P1 copies), y only
  // [r]_2 (P0, P2 copies), so P1's and P2's cross terms vanish and P0's sums are single Grams.
  const bool bit_form = !ys && x.c[0] && !x.c[1] && !x.c[2] && x.c[3] && !x.c[4] && !x.c[5] &&
                        !y.c[0] && y.c[1] && !y.c[2] && !y.c[3] && !y.c[4] && y.c[5];
  if (ys) {
    CK(cudaMemsetAsync(s.S, 0, 4 * 192 * 8, st));
    launch_gram_lifted(st, x.c, ys->c, Dh, D, s.S);   // S00 | S01 + S10 | 0 | S11
  } else if (bit_form) {
    // G00, G11 and G(x0 + x1, y0 + y1); G01 + G10 = G(x0 + x1, y0 + y1) - G00 - G11
    CK(cudaMemsetAsync(s.Pmat, 0, 3 * 4096 * 8, st));
    CK(cudaMemsetAsync(s.S, 0, 4 * 192 * 8, st));
    bool done = false;
    if (ctx->gemm_path == MPC_GEMM_LIMB_TC) {
      // tensor cores: G00, G11 and the cross sum G01 + G10 directly
      g_launches += 1;
      {
        Phase kp(ctx, MPC_PROF_K_GRAM, 4.0 * Dh * 4096);
        done = gram3_tc(st, Dh, x.c[0], y.c[1], s.Pmat, ctx->status, ST_TIMEOUT,
                        ctx->tune.gram_split) == 0;
      }
      if (done) {
        launch_gr_fold_reduce(st, s.Pmat, 3, s.aux);
        CK(cudaMemcpyAsync(S00, s.aux, 512, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(S11, s.aux + 64, 512, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(S01, s.aux + 128, 512, cudaMemcpyDeviceToDevice, st));
      } else {
        g_launches -= 1;
      }
    }
    if (!done) {
      gram(ctx, s.Pmat, x.c[0], nullptr, 1, 128, y.c[1], nullptr, 1, 128, Dh, 1);
      gram(ctx, s.Pmat + 4096, x.c[0] + 64, nullptr, 1, 128, y.c[1] + 64, nullptr, 1, 128, Dh, 1);
      gram(ctx, s.Pmat + 8192, x.c[0], x.c[0] + 64, 1, 128, y.c[1], y.c[1] + 64, 1, 128, Dh, 1);
      launch_gr_fold_reduce(st, s.Pmat, 3, s.aux);            // aux: G00, G11, Gsum (64 each)
      CK(cudaMemcpyAsync(S00, s.aux, 512, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(S11, s.aux + 64, 512, cudaMemcpyDeviceToDevice, st));
      launch_gr_lincomb(st, ctx->cst + CST_ONE, s.aux + 128, ctx->cst + CST_MONE, s.aux, s.aux + 192);
      launch_gr_lincomb(st, ctx->cst + CST_ONE, s.aux + 192, ctx->cst + CST_MONE, s.aux + 64, S01);
    }
  } else {
    bool done = false;
    if (ctx->gemm_path == MPC_GEMM_LIMB_TC) {
      // tensor cores: the party sums of S00, S11 and S01 + S10 as Gram blocks (in S01; S10 = 0),
      // one job per Gram term.  P0: G(x0 + x1, y0 + y1); P1: -G(x2, y3) - G(y2, x3);
      // P2: G(x4, y4 - y5) - G(y4, x5).  A term with an absent first source takes the second's
      // scale into its sign; a term with an absent side is zero.
      const u64 M1 = ~0ull;
      GramJobs jobs{};
      jobs.off_x = 3 * 4096;
      jobs.off_oo = 9 * 4096;
      auto add = [&](int party, const u64* a0, const u64* a1, u64 sa1, const u64* b0,
                     const u64* b1, u64 sb1, u64 sign) {
        if (!a0) { a0 = a1; a1 = nullptr; sign *= sa1; }
        if (!b0) { b0 = b1; b1 = nullptr; sign *= sb1; }
        if (!a0 || !b0) return;
        jobs.j[jobs.n++] = GramJob{a0, a1, sa1, b0, b1, sb1, s.Pmat + party * 4096, sign};
      };
      add(0, x.c[0], x.c[1], 1, y.c[0], y.c[1], 1, 1);
      add(1, x.c[2], nullptr, 0, y.c[3], nullptr, 0, M1);
      add(1, y.c[2], nullptr, 0, x.c[3], nullptr, 0, M1);
      add(2, x.c[4], nullptr, 0, y.c[4], y.c[5], M1, 1);
      add(2, y.c[4], nullptr, 0, x.c[5], nullptr, 0, M1);
      CK(cudaMemsetAsync(s.Pmat, 0, 12 * 4096 * 8, st));
      int nl = 0;
      for (int q = 0; q < jobs.n; ++q) nl |= (jobs.j[q].a1 || jobs.j[q].b1) ? 2 : 1;
      nl = (nl & 1) + (nl >> 1);   // one launch for the single-source jobs, one for the others
      g_launches += nl;
      {
        Phase kp(ctx, MPC_PROF_K_GRAM, 4.0 * Dh * 4096 * jobs.n);
        done = gram_jobs_tc(st, Dh, jobs, ctx->status, ST_TIMEOUT, ctx->tune.gram_split) == 0;
      }
      if (done) {
        launch_gr_fold_reduce(st, s.Pmat, 12, s.S);   // S00 | S01 + S10 | 0 | S11
      } else {
        g_launches -= nl;
      }
    }
    if (!done) {
      if ((rc = party_sums(ctx, f[0], g[0], Dh, s.Pmat, S00))) return rc;
      if ((rc = party_sums(ctx, f[0], g[1], Dh, s.Pmat + 3 * 4096, S01))) return rc;
      if ((rc = party_sums(ctx, f[1], g[0], Dh, s.Pmat + 6 * 4096, S10))) return rc;
      if ((rc = party_sums(ctx, f[1], g[1], Dh, s.Pmat + 9 * 4096, S11))) return rc;
    }
  }
  round_tail(ctx, vid, batch, k, z, zo, s);
  // f(zeta) = f(0) + zeta (f(1) - f(0)): rows [x_{2i+1} - x_{2i}] times M_zeta, plus x_{2i}.
  // Vectors that sit at one stride (the dense plans put a slot's x vectors, then its y vectors,
  // one after another) go through one launch: segment s of Dh rows (padded to whole tiles); all
  // of them when x's and y's rows have the same capacity, else each side's.  Only short vectors
  // are batched: there one launch replaces several latency-bound ones, while on long ones the
  // segment arithmetic of the batched row map costs more than the launches it saves.
  auto fold_batched = [&](const u64* const* ins, u64* const* outs, int n) -> bool {
    if (ctx->gemm_path != MPC_GEMM_LIMB_TC || Dh > ctx->tune.fold_batch_max || n < 2) return false;
    const long long sin = ins[1] - ins[0], sout = outs[1] - outs[0];
    for (int i = 1; i < n; ++i)
      if (ins[i] - ins[0] != i * sin || outs[i] - outs[0] != i * sout) return false;
    if (sin <= 0 || sout <= 0) return false;
    const long long Rp = (Dh + 127) / 128 * 128;
    GrMMArgs g = grargs(ctx);
    g.R = n * Rp;
    g.p0 = ins[0] + 64;
    g.p1 = ins[0];
    g.s1 = ~0ull;
    g.in = GrRowMap{Rp, 128, sin};
    g.qvalid = Dh;
    g.Mmat = s.MM;
    g.add0 = ins[0];
    g.add0_in = 1;
    g.out = outs[0];
    g.om = GrRowMap{Rp, 64, sout};
    g_launches += 1;
    Phase kp(ctx, MPC_PROF_K_GR_MATMUL, (double)n * Dh * 4096);
    if (gr_matmul_tc_ex(st, g, ctx->status, ST_TIMEOUT) == 0) return true;
    g_launches -= 1;
    return false;
  };
  const u64* ins[12];
  u64* outs[12];
  int nx = 0, n = 0;
  for (int side = 0; side < (ys ? 1 : 2); ++side)
    for (int c = 0; c < 6; ++c) {
      const u64* in = side ? y.c[c] : x.c[c];
      if (!in) continue;
      ins[n] = in;
      outs[n] = side ? yo.c[c] : xo.c[c];
      ++n;
      if (!side) ++nx;
    }
  bool done_all = fold_batched(ins, outs, n);
  for (int side = 0; side < (ys ? 1 : 2) && !done_all; ++side) {
    const int i0 = side ? nx : 0, i1 = side ? n : nx;
    if (fold_batched(ins + i0, outs + i0, i1 - i0)) continue;
    for (int i = i0; i < i1; ++i)
      if ((rc = gr_matmul(ctx, Dh, ins[i] + 64, ins[i], ~0ull, 128, s.MM, ins[i], 128, outs[i], 64)))
        return rc;
  }
  if (ys)   // the fold element is the first GR element of the Lagrange coefficients
    for (int c = 0; c < 6; ++c)
      if (ys->c[c]) launch_fold_lifted(st, ys->c[c], Dh, D, s.coef, yo.c[c]);
  trace_round(ctx, trace, k, s);
  return cuda_check(ctx, "reduce_round");
}

// Pi_InnerVerify (Fig. DPV) on a dense claim of dimension D.
int inner_verify_dense(mpc_ctx* ctx, u64 vid, u32 batch, const Vec& x, const Vec& y, long long D,
                       const u64* z, const Small& s, const IVBuf& b, u64* trace, int R) {
  cudaStream_t st = ctx->st;
  const u64 obj = make_obj(vid, batch, 0);
  const long long w = (D + 1) * 64;
  const u64 M1 = ~0ull;
  // alpha random, not revealed
  launch_gr_random_shared(st, 1, ctx->k01, ctx->k02, ctx->k12, P_VER_ALPHA, obj, s.alpha);
  const u64* a = s.alpha;
  // multiplication matrices: r_a = a0 + a1 (P0), a3 (P1's [r]_1), a2 (P1's m),
  // a4 - a5 (P2's m - [r]_2), a4 (P2's m)
  u64* ra = s.aux;
  u64* d45 = s.aux + 64;
  launch_gr_lincomb(st, ctx->cst + CST_ONE, a, ctx->cst + CST_ONE, a + 64, ra);
  launch_gr_lincomb(st, ctx->cst + CST_ONE, a + 256, ctx->cst + CST_MONE, a + 320, d45);
  launch_gr_mulmat2(st, ra, a + 192, s.MA);            // MA[0] = M(r_a), MA[1] = M(a3)
  launch_gr_mulmat2(st, a + 128, d45, s.MA + 8192);    // MA[2] = M(a2), MA[3] = M(a4 - a5)
  launch_gr_mulmat2(st, a + 256, nullptr, s.MA + 16384);  // MA[4] = M(a4)
  CK(cudaMemsetAsync(b.zero, 0, (size_t)w * 8, st));
  auto comp = [&](int c) -> const u64* { return x.c[c] ? x.c[c] : b.zero; };
  // masks of x' = x alpha (words i*64 + c of the (P_VER_XA, R1/R2) streams)
  launch_fill_masks(st, w, ctx->k01, ctx->k02, P_VER_XA, obj, b.xp);
  {  // P0: Gamma_i = r_{x_i} r_a + [r_{x'_i}]_1 + [r_{x'_i}]_2, message [Gamma]_2 = Gamma - [Gamma]_1
    GemmTerm T;
    T.A = op(comp(0), 64, 0, x.c[1], 1);
    T.B = op(s.MA, 64);
    Epi e = epi_store(b.g2o, 64);
    e.add0 = b.xp;
    e.add1 = b.xp + w;
    e.prf_sign = M1;
    e.key = ctx->k01;
    e.tag = make_tag(P_VER_XA, C_G1);
    e.obj = obj;
    gemm_u64_small(st, D, 64, 64, 1, &T, e);
  }
  int rc;
  if ((rc = deliver(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, b.g2o, b.g2i, D * 64, -1))) return rc;
  {  // P1: [m]_1 = -(m_x [r_a]_1 + m_a [r_x]_1) + [Gamma]_1
    GemmTerm T[2];
    T[0].A = op(comp(2), 64);
    T[0].B = op(s.MA + 4096, 64);
    T[1].A = op(comp(3), 64);
    T[1].B = op(s.MA + 8192, 64);
    Epi e = epi_store(b.p1o, 64);
    e.acc_sign = M1;
    e.prf_sign = 1;
    e.key = ctx->k01;
    e.tag = make_tag(P_VER_XA, C_G1);
    e.obj = obj;
    gemm_u64_small(st, D, 64, 64, 2, T, e);
  }
  {  // P2: [m]_2 = m_x (m_a - [r_a]_2) - [r_x]_2 m_a + [Gamma]_2
    GemmTerm T[2];
    T[0].A = op(comp(4), 64);
    T[0].B = op(s.MA + 12288, 64);
    T[1].A = op(comp(5), 64, 0, nullptr, 1, M1);
    T[1].B = op(s.MA + 16384, 64);
    Epi e = epi_store(b.p2o, 64);
    e.add0 = b.g2i;
    gemm_u64_small(st, D, 64, 64, 2, T, e);
  }
  if ((rc = deliver(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, b.p1o, b.p2i, D * 64, -1))) return rc;
  if ((rc = deliver(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, b.p2o, b.p1i, D * 64, -1))) return rc;
  launch_exchange_finish(st, w, b.p1o, b.p1i, b.p2o, b.p2i, b.xp, -1, nullptr);
  // x'' = [x'_0 .. x'_{D-1}, alpha]; y'' = [y_0 .. y_{D-1}, -z]
  for (int c = 0; c < 6; ++c) {
    CK(cudaMemcpyAsync(b.xp + c * w + D * 64, a + c * 64, 512, cudaMemcpyDeviceToDevice, st));
    if (y.c[c])
      CK(cudaMemcpyAsync(b.yy + c * w, y.c[c], (size_t)D * 512, cudaMemcpyDeviceToDevice, st));
    else
      CK(cudaMemsetAsync(b.yy + c * w, 0, (size_t)D * 512, st));
    launch_neg_copy(st, z + c * 64, 64, b.yy + c * w + D * 64);
  }
  View u, v;
  for (int c = 0; c < 6; ++c) {
    u.c[c] = b.xp + c * w;
    v.c[c] = b.yy + c * w;
  }
  u.ld = 64;
  v.ld = 64;
  if ((rc = party_sums(ctx, u, v, D + 1, s.Pmat, s.Sfull))) return rc;
  inner_finish(ctx, s.Sfull, P_VER_DELTA, obj, s.tmp6);
  rec1(ctx, s.tmp6, b.delta);
  launch_gr_check_zero(st, b.delta, ctx->status, ST_VERIFY);
  if (trace)
    CK(cudaMemcpyAsync(trace + (long long)R * TRACE_ROUND, b.delta, 512, cudaMemcpyDeviceToDevice, st));
  return cuda_check(ctx, "inner_verify");
}

// Dense rounds k = k0..R followed by Pi_InnerVerify.
// ylift (optional): the y vectors entering round k0 are lifted ring words (one word per element
// and present component); they are folded into dv.y's GR rows by the first round, or lifted there
// when no round is left.
int run_dense(mpc_ctx* ctx, u64 vid, u32 batch, Dense& dv, long long D, const u64* z0, int k0,
              int R, const Small& s, const IVBuf& ivb, u64* trace, const Vec* ylift = nullptr) {
  int rc;
  const u64* z = z0;
  int zi = 0;
  for (int k = k0; k <= R; ++k) {
    Vec& x = dv.x[dv.cur];
    Vec& y = dv.y[dv.cur];
    Vec& xo = dv.x[dv.cur ^ 1];
    Vec& yo = dv.y[dv.cur ^ 1];
    u64* zo = s.z[zi];
    if ((rc = reduce_round_dense(ctx, vid, batch, k, x, y, D, z, xo, yo, zo, s, trace,
                                 k == k0 ? ylift : nullptr)))
      return rc;
    z = zo;
    zi ^= 1;
    dv.cur ^= 1;
    D = (D + 1) / 2;
  }
  if (ylift && k0 > R)
    for (int c = 0; c < 6; ++c)
      if (ylift->c[c]) launch_gr_lift(ctx->st, ylift->c[c], D, dv.y[dv.cur].c[c]);
  return inner_verify_dense(ctx, vid, batch, dv.x[dv.cur], dv.y[dv.cur], D, z, s, ivb, trace, R);
}

long long dim_after(long long D, int R) {
  for (int k = 0; k < R; ++k) D = (D + 1) / 2;
  return D;
}

// Allocate ping-pong vectors for a dense claim of dimension D over the present components.  With
// ylifted_R >= 1 the y side enters in ring words (run_dense's ylift) and the first round writes
// slot 1, so slot 0 of y only ever holds the outputs of round 2 and later (at most cap[1] rows).
// With x_from_bits the first round writes x's slot 1 without reading slot 0 (the edaBit
// inner-product batch), so x's slot 0 is half size as well.
Dense plan_dense(Arena& a, long long D, const bool xc[6], const bool yc[6], int ylifted_R = 0,
                 bool x_from_bits = false) {
  Dense d;
  d.cap[0] = D + 1;
  d.cap[1] = (D + 1) / 2 + 1;
  const long long ycap0 = ylifted_R >= 1 ? d.cap[1] : d.cap[0];
  const long long xcap0 = x_from_bits && ylifted_R >= 1 ? d.cap[1] : d.cap[0];
  // a slot's x vectors, then its y vectors: each side's present vectors sit at one stride (the
  // batched folds use that)
  for (int i = 0; i < 2; ++i) {
    for (int c = 0; c < 6; ++c) d.x[i].c[c] = xc[c] ? a.take<u64>((i ? d.cap[1] : xcap0) * 64) : nullptr;
    for (int c = 0; c < 6; ++c)
      d.y[i].c[c] = yc[c] ? a.take<u64>((i ? d.cap[1] : ycap0) * 64) : nullptr;
  }
  return d;
}

// Reads the status word after a verification; the products under pend_key leave the pending
// set only on a clean status (after a failure the context is aborted for good).
int finish_verify(mpc_ctx* ctx, u64 pend_key) {
  u32 stv = 0;
  int rc = read_status(ctx, &stv);
  if (rc) return rc;
  if (!(stv & (ST_ABORT | ST_VERIFY))) ctx->pending.erase(pend_key);
  if (stv & ST_ABORT) {
    ctx->aborted = true;
    return fail(ctx, MPC_ERR_ABORT, "Pi_Rec: inconsistent messages");
  }
  if (stv & ST_VERIFY) {
    ctx->aborted = true;
    return fail(ctx, MPC_ERR_VERIFY, "verification failed: Delta != 0");
  }
  return MPC_OK;
}

// ---- plans ----------------------------------------------------------------------------------
struct MatmulPlan {
  u64 *g2o, *g2i, *mz1, *mz2, *mz1i, *mz2i;
  u64 *gp2, *gq2, *gp2i, *gq2i, *mp1, *mq1, *mpi1, *mqi1, *mpi2, *mqi2;
  void* tc;   // digit planes of the tensor-core path (null on the u64 path)
};

MatmulPlan plan_matmul(Arena& a, long long M, long long N, long long K, bool trunc, bool tc) {
  const long long E = M * N;
  MatmulPlan p{};
  p.tc = tc ? (void*)a.take<unsigned char>((long long)limb_tc_scratch_bytes(M, N, K, 2)) : nullptr;
  p.g2o = a.take<u64>(E); p.g2i = a.take<u64>(E);
  p.mz1 = a.take<u64>(E); p.mz2 = a.take<u64>(E);
  p.mz1i = a.take<u64>(E); p.mz2i = a.take<u64>(E);
  if (trunc) {
    p.gp2 = a.take<u64>(E); p.gq2 = a.take<u64>(E);
    p.gp2i = a.take<u64>(E); p.gq2i = a.take<u64>(E);
    p.mp1 = a.take<u64>(E); p.mq1 = a.take<u64>(E);
    p.mpi1 = a.take<u64>(E); p.mqi1 = a.take<u64>(E);
    p.mpi2 = a.take<u64>(E); p.mqi2 = a.take<u64>(E);
  }
  return p;
}

struct RecPlan {
  u64 *in_p2_r1, *in_p1_r2, *in_p0_m, *out_dev;
  u32* hs[6];
  u32* dg;   // 6 x 8
};

RecPlan plan_rec(Arena& a, long long n, bool need_out) {
  RecPlan p{};
  p.in_p2_r1 = a.take<u64>(n);
  p.in_p1_r2 = a.take<u64>(n);
  p.in_p0_m = a.take<u64>(n);
  for (int i = 0; i < 6; ++i) p.hs[i] = a.take<u32>((long long)hash_scratch_words(n));
  p.dg = a.take<u32>(48);
  p.out_dev = need_out ? a.take<u64>(n) : nullptr;
  return p;
}

// A table of powers r^i, i < n (rows of 64 words): rows below L by repeated multiplication, row
// h L + l (h >= 1) = r^(hL) r^l, all of them one grouped GR-matrix product (matrix h - 1 for the
// rows L h .. L h + L - 1).  L is a multiple of 128 near sqrt(n).
struct PowPlan {
  long long n, L, nhi;
  u64* Thi;   // r^(hL), h < nhi
  u64* Mhi;   // multiplication matrices of r^(hL), h = 1 .. nhi - 1
};

PowPlan plan_pow(Arena& a, long long n) {
  PowPlan p;
  p.n = n;
  long long L = 1024;
  while (L * L < n) L += 128;
  p.L = L;
  p.nhi = (n + L - 1) / L;
  p.Thi = a.take<u64>(p.nhi * 64);
  p.Mhi = a.take<u64>(std::max<long long>(p.nhi - 1, 1) * 4096);
  return p;
}

// table[i] = r^i for i < p.n; aux: 64 words of scratch
int power_table(mpc_ctx* ctx, const u64* r, const PowPlan& p, u64* table, u64* aux) {
  cudaStream_t st = ctx->st;
  if (ctx->gemm_path != MPC_GEMM_LIMB_TC || p.nhi <= 1) {
    launch_gr_powers(st, r, p.n, table);
    return MPC_OK;
  }
  launch_gr_powers(st, r, p.L, table);
  launch_gr_mul1(st, table + (p.L - 1) * 64, r, aux);                 // r^L
  launch_gr_powers(st, aux, p.nhi, p.Thi);
  launch_gr_mulmat_batch(st, p.nhi - 1, p.Thi + 64, 64, p.Mhi);
  GrMMArgs g = grargs(ctx);
  g.R = (p.nhi - 1) * p.L;
  g.p0 = table;
  g.in = GrRowMap{p.L, 64, 0};
  g.Mmat = p.Mhi;
  g.mrows = p.L;
  g.out = table + p.L * 64;
  g.om = GrRowMap{0, 64, 0};
  g.out_lim = (p.n - p.L) * 64;
  g_launches += 1;
  Phase kp(ctx, MPC_PROF_K_GR_MATMUL, (double)(p.n - p.L) * 4096);
  if (gr_matmul_tc_ex(st, g, ctx->status, ST_TIMEOUT) == 0) return MPC_OK;
  g_launches -= 1;
  launch_gr_powers(st, r, p.n, table);
  return MPC_OK;
}

struct VMultPlan {
  Small s;
  u64* pw;
  PowPlan pp;
  Dense dv;
  IVBuf iv;
  int R;
};

VMultPlan plan_vmult(Arena& a, long long n, int R) {
  VMultPlan p;
  p.R = R < 0 ? default_R(n) : R;
  p.s = plan_small(a);
  p.pw = a.take<u64>(n * 64);
  p.pp = plan_pow(a, n);
  const bool all[6] = {true, true, true, true, true, true};
  p.dv = plan_dense(a, n, all, all, p.R);
  p.iv = plan_iv(a, dim_after(n, p.R));
  return p;
}

// deferred Pi_MultVerify over several calls: the gathered triples, then the verification plan
struct VMultCallsPlan {
  u64 *x, *y, *z;
  VMultPlan v;
};

VMultCallsPlan plan_vmult_calls(Arena& a, long long n, int R) {
  VMultCallsPlan p;
  p.x = a.take<u64>(6 * n);
  p.y = a.take<u64>(6 * n);
  p.z = a.take<u64>(6 * n);
  p.v = plan_vmult(a, n, R);
  return p;
}

// One verification chunk of the truncation batch (E consecutive outputs of the layer).
struct TruncPlan {
  long long E = 0;
  int R1 = 0, kd = 0;
  long long Dt = 0;
  long long L = 0, Epad = 0, nhi = 0;   // S = sum over e_hi < nhi of T_hi (x) (sum over e_lo < L ...)
  u64 *b1, *b2, *Rtab, *S, *Zpq, *V, *W, *hsum, *S3, *zt, *S_hi, *Pst, *Thi, *Mhi;
  u64 *B1T, *B2T;   // bit-transposed b1, b2: [j][e / 64]
  unsigned char* TL8;
  // tensor-core materialisation with r^(2e) = r^(2 Lm e_hi) r^(2 e_lo), e = e_hi Lm + e_lo:
  // Tm[e_lo][j] = r^(2 e_lo) (-V_j), Bm[e_hi] = M(r^(2 Lm e_hi)), Vm[j] = M(-V_j), bT = b1 in
  // (e_lo, e_hi) order (nhm x Lm view transposed)
  long long Lm = 0, nhm = 0;
  u64 *Tm = nullptr, *Bm = nullptr, *Vm = nullptr, *bT = nullptr;
  // compact table (E a multiple of L on that path): only r^(2 e_lo), e_lo < L, is materialised;
  // sum_e r^(2e) pq_c[e] = sum_{e_hi} T_hi[e_hi] (sum_{e_lo} pq_c[e] r^(2 e_lo)) (a limb GEMM over
  // the first block, then 12 nhi GR products), and the rows r^(2 Lm e_hi) come from T_hi x r^(2 e_lo)
  bool compact = false;
  bool tc_combine = false;   // sum_{e_hi} T_hi (x) S_hi on the tensor cores
  u64 *Zhi = nullptr, *Zrep = nullptr, *Zprod = nullptr, *Prow = nullptr;
  u64* pqc = nullptr;        // the chunk's 12 rows of <p>, <q> gathered (chunked batches only)
  Dense dt;
  IVBuf ivt;
};

// A truncation batch of E outputs: nchunks chunks of C outputs (the last one ragged).
struct TruncBatch {
  long long E = 0, nchunks = 0, C = 0;
  TruncPlan tp[2];   // plans of a full chunk and of the ragged last one
};

struct VMatPlan {
  Small s;
  u64 *Q, *P, *T, *Pz;
  Dense dv;
  IVBuf iv;
  int R0;
  bool trunc = false;
  TruncBatch tb;
  void* tcs = nullptr;            // tensor-core digit planes (limb path only)
};

// Layout decisions of a truncation chunk of E outputs (no allocation).
struct TruncShape {
  long long L, Epad, nhi, Lm = 0, nhm = 0;
  int R1, kd;
  bool compact = false, tc_combine = false, blocked = false;
};

TruncShape trunc_shape(long long E, int R1, bool tc, const mpc_tuning& tu) {
  TruncShape h;
  h.R1 = R1 < 0 ? default_R(64 * E) : R1;
  h.kd = std::min(h.R1, 6);
  const long long Lb = tu.trunc_block;
  h.blocked = E >= Lb;
  h.L = h.blocked ? Lb : ((E + 127) / 128) * 128;
  h.Epad = ((E + h.L - 1) / h.L) * h.L;
  h.nhi = h.Epad / h.L;
  h.compact = tc && h.kd == 6 && h.blocked && E % h.L == 0;
  h.tc_combine = tc && h.nhi >= tu.tc_combine_min;
  if (tc && h.kd == 6 && h.blocked) {
    if (tu.row_split > 0) {
      // at most E rounded up to a tile: the row-split table reads r^(2 e_lo) for e_lo < Lm
      h.Lm = std::min<long long>(tu.row_split, (E + 127) / 128 * 128);
      h.nhm = ((E + h.Lm - 1) / h.Lm + 127) / 128 * 128;
    } else {
      // Lm = 128 a with a odd near sqrt(E) / 128, and nhm = 128 b >= E / Lm with the fewest rows
      // past E: the bit product writes its rows Lm rows apart, and a stride of a multiple of
      // 2 MB (a even at E = 2^24) puts a tile's 128 rows on the same memory channels
      long long sq = 1;
      while (sq * sq < E) ++sq;
      const long long a0 = (sq + 127) / 128;
      h.Lm = 128 * a0;
      h.nhm = ((E + h.Lm - 1) / h.Lm + 127) / 128 * 128;
      if (a0 >= 4) {   // strides of 512 KB and more
        long long best = -1;
        for (long long aa = (a0 * 3 / 4) | 1; aa <= 2 * a0 + 1; aa += 2) {
          const long long bb = (E + 128 * 128 * aa - 1) / (128 * 128 * aa);
          const long long rows = 128 * 128 * aa * bb;
          if (best < 0 || rows < h.Lm * h.nhm ||
              (rows == h.Lm * h.nhm && std::llabs(aa - a0) < std::llabs(best - a0))) {
            best = aa;
            h.Lm = 128 * aa;
            h.nhm = 128 * bb;
          }
        }
      }
    }
    // the compact table keeps r^(2 e_lo) for e_lo < L only, and the row-split table reads e_lo < Lm
    if (h.Lm > h.L) h.compact = false;
  }
  return h;
}

// tensor-core scratch of a truncation chunk: the S_hi combination (64 x 262144 x nhi) and the
// compact table's sum over the first block (12 nhi x 64 x L)
size_t trunc_tc_scratch(const TruncShape& h) {
  size_t b = 0;
  if (h.tc_combine) b = std::max(b, limb_tc_scratch_bytes(64, 262144, h.nhi, 1));
  if (h.compact) b = std::max(b, limb_tc_scratch_bytes(12 * h.nhi, 64, h.L, 1));
  return b;
}

TruncPlan plan_trunc(Arena& a, long long E, int R1, bool tc, bool chunked, const mpc_tuning& tu) {
  TruncPlan p;
  const TruncShape h = trunc_shape(E, R1, tc, tu);
  p.E = E;
  p.R1 = h.R1;
  p.kd = h.kd;
  p.Dt = E * (64 >> p.kd);
  p.L = h.L;
  p.Epad = h.Epad;
  p.nhi = h.nhi;
  p.compact = h.compact;
  p.tc_combine = h.tc_combine;
  p.b1 = a.take<u64>(p.Epad);
  p.b2 = a.take<u64>(p.Epad);
  p.Rtab = a.take<u64>((p.compact ? p.L : p.Epad) * 64);
  p.S = a.take<u64>(4096 * 64);
  p.TL8 = a.take<unsigned char>(1024 * p.L);
  p.B1T = a.take<u64>(p.Epad);
  p.B2T = a.take<u64>(p.Epad);
  p.S_hi = a.take<u64>(p.nhi * 4096 * 64);
  p.Pst = a.take<u64>(64ll * 262144);
  p.Thi = a.take<u64>(p.nhi * 64);
  p.Mhi = a.take<u64>(std::max<long long>(1, p.nhi - 1) * 4096);
  p.Zpq = a.take<u64>(12 * 64);
  p.V = a.take<u64>(4096);
  p.W = a.take<u64>(4096);
  p.hsum = a.take<u64>(128);
  p.S3 = a.take<u64>(2 * 192);
  p.zt = a.take<u64>(2 * 384);
  if (chunked) p.pqc = a.take<u64>(12 * E);
  if (h.Lm) {
    p.Lm = h.Lm;
    p.nhm = h.nhm;
    p.Tm = a.take<u64>(p.Lm * 4096);
    p.Bm = a.take<u64>((E + p.Lm - 1) / p.Lm * 4096);
    if (p.compact) {
      p.Zhi = a.take<u64>(12 * p.nhi * 64);
      p.Zrep = a.take<u64>(12 * p.nhi * 64);
      p.Zprod = a.take<u64>(12 * p.nhi * 64);
      p.Prow = a.take<u64>(3 * ((E + p.Lm - 1) / p.Lm) * 64);
    }
    p.Vm = a.take<u64>(64 * 4096);
    p.bT = a.take<u64>(p.nhm * p.Lm);
  }
  const bool xc[6] = {true, false, false, true, false, false};
  const bool yc[6] = {false, true, false, false, false, true};
  p.dt = plan_dense(a, p.Dt, xc, yc);
  p.ivt = plan_iv(a, dim_after(p.Dt, p.R1 - p.kd));
  return p;
}

// Chunks of the truncation batch of E outputs: n chunks of C outputs, the last E - (n-1) C.
void trunc_chunks(long long E, const mpc_tuning& tu, long long* n, long long* C) {
  *C = std::min<long long>(E, tu.trunc_chunk);
  *n = (E + *C - 1) / *C;
}
constexpr long long MAX_TRUNC_CHUNKS = 15;   // batch ids 1 .. 15 of the object-id layout

// Tensor-core scratch of a truncation batch of E outputs (the larger of its two chunk shapes);
// -1 when it has more than MAX_TRUNC_CHUNKS chunks.
long long trunc_batch_tcs(long long E, int R1, bool tc, const mpc_tuning& tu) {
  long long n = 0, C = 0;
  trunc_chunks(E, tu, &n, &C);
  if (n > MAX_TRUNC_CHUNKS) return -1;
  const long long Elast = E - (n - 1) * C;
  return (long long)std::max(trunc_tc_scratch(trunc_shape(C, R1, tc, tu)),
                             trunc_tc_scratch(trunc_shape(Elast, R1, tc, tu)));
}

// The chunks run one after another: their plans share the rest of the workspace.
void plan_trunc_batch(Arena& a, long long E, int R1, bool tc, const mpc_tuning& tu,
                      TruncBatch& b) {
  b.E = E;
  trunc_chunks(E, tu, &b.nchunks, &b.C);
  const long long Elast = E - (b.nchunks - 1) * b.C;
  const bool chunked = b.nchunks > 1;
  const size_t off0 = a.off;
  b.tp[0] = plan_trunc(a, b.C, R1, tc, chunked, tu);
  const size_t off1 = a.off;
  if (Elast != b.C) {
    a.off = off0;
    b.tp[1] = plan_trunc(a, Elast, R1, tc, chunked, tu);
    a.off = std::max(off1, a.off);
  } else {
    b.tp[1] = b.tp[0];
  }
}

// false when the layer cannot be planned (too many truncation chunks)
bool plan_vmat(Arena& a, long long M, long long N, long long K, int t, int R0, int R1, bool tc,
               const mpc_tuning& tu, VMatPlan& p) {
  p.R0 = R0 < 0 ? default_R(K) : R0;
  p.s = plan_small(a);
  p.trunc = t >= 0;
  const long long E = M * N;
  long long trunc_tcs = 0;
  if (p.trunc && (trunc_tcs = trunc_batch_tcs(E, R1, tc, tu)) < 0) return false;
  // digit planes of the batch-0 products (X^T P, W Q, Z Q) and of the truncation chunks'
  // tensor-core products, on the tensor-core path
  p.tcs = tc ? (void*)a.take<unsigned char>((long long)std::max(
                   {limb_tc_scratch_bytes(K, 64, M, 1), limb_tc_scratch_bytes(K, 64, N, 1),
                    limb_tc_scratch_bytes(6 * M, 64, N, 1), (size_t)trunc_tcs}))
             : nullptr;
  p.Q = a.take<u64>(N * 64);
  p.P = a.take<u64>(M * 64);
  p.T = a.take<u64>(6 * M * 64);
  p.Pz = a.take<u64>(6 * 4096);
  const bool all[6] = {true, true, true, true, true, true};
  p.dv = plan_dense(a, K, all, all);
  p.iv = plan_iv(a, dim_after(K, p.R0));
  if (p.trunc) plan_trunc_batch(a, E, R1, tc, tu, p.tb);
  return true;
}

// plan of a standalone truncation batch's verification (mpc_verify_trunc)
struct VTruncPlan {
  Small s;
  TruncBatch tb;
  void* tcs = nullptr;
};

bool plan_vtrunc(Arena& a, long long n, int R, bool tc, const mpc_tuning& tu, VTruncPlan& p) {
  const long long tcs = trunc_batch_tcs(n, R, tc, tu);
  if (tcs < 0) return false;
  p.s = plan_small(a);
  p.tcs = tc && tcs > 0 ? (void*)a.take<unsigned char>(tcs) : nullptr;
  plan_trunc_batch(a, n, R, tc, tu, p.tb);
  return true;
}

// One chunk of batch 1 of Pi_BIVerify (Fig. PBDP): the 2 E inner products of the truncation pairs
// of outputs e0 .. e0 + E - 1 (E = p.E) of a layer of E_all outputs, with the challenge and round
// streams of batch `batch`.  pq_all: the layer's 12 rows of <p>, <q> (stride E_all).
int verify_trunc_chunk(mpc_ctx* ctx, TruncPlan& p, const Small& s, void* tcs, const u64* pq_all,
                       long long E_all, long long e0, int trunc_bits, u64 verify_id, u32 batch,
                       u64 matmul_call_id, u64* tr, const u64* row_keys, long long N) {
  cudaStream_t st = ctx->st;
  Phase* phase = new Phase(ctx, MPC_PROF_TRUNC_SETUP);
  const u64 mobj = make_obj(matmul_call_id, 0, 0);
  const long long E = p.E;
  int rc;
  if (p.pqc)   // this chunk's outputs of the 12 rows of <p>, <q>, gathered to a stride of E
    CK(cudaMemcpy2DAsync(p.pqc, (size_t)E * 8, pq_all + e0, (size_t)E_all * 8, (size_t)E * 8, 12,
                         cudaMemcpyDeviceToDevice, st));
  const u64* pq = p.pqc ? p.pqc : pq_all;
  reveal(ctx, P_VER_R, make_obj(verify_id, batch, 0), s.tmp6, s.r);
  launch_trunc_u(st, s.r, trunc_bits, p.V);                         // V_j = u_j
  for (int j = 0; j < 64; ++j)
    CK(cudaMemcpyAsync(p.W + j * 64, ctx->cst + CST_ONE, 512, cudaMemcpyDeviceToDevice, st));
  if (p.Epad > E) {
    CK(cudaMemsetAsync(p.b1 + E, 0, (size_t)(p.Epad - E) * 8, st));
    CK(cudaMemsetAsync(p.b2 + E, 0, (size_t)(p.Epad - E) * 8, st));
  }
  if (row_keys) {
    launch_prf_words_keyed(st, E, ctx->k01, make_tag(P_TRUNC_BITS, C_TB1), row_keys, N, p.b1, e0);
    launch_prf_words_keyed(st, E, ctx->k02, make_tag(P_TRUNC_BITS, C_TB2), row_keys, N, p.b2, e0);
  } else {
    launch_prf_words(st, E, ctx->k01, make_tag(P_TRUNC_BITS, C_TB1), mobj, p.b1, e0);
    launch_prf_words(st, E, ctx->k02, make_tag(P_TRUNC_BITS, C_TB2), mobj, p.b2, e0);
  }
  launch_gr_mul1(st, s.r, s.r, s.aux + 64);                          // r^2
  // r^(2e) for e < Epad: r^(2 e_lo) for e_lo < L by repeated multiplication, then every further
  // block of L rows is that block times the constant r^(2 L e_hi) (a 64 x 64 matrix product)
  launch_gr_powers(st, s.aux + 64, p.L, p.Rtab);
  if (p.compact) {
    launch_gr_mul1(st, p.Rtab + (p.L - 1) * 64, s.aux + 64, s.aux + 128);   // r^(2L)
    launch_gr_powers(st, s.aux + 128, p.nhi, p.Thi);
  } else if (p.nhi > 1) {
    launch_gr_mul1(st, p.Rtab + (p.L - 1) * 64, s.aux + 64, s.aux + 128);   // r^(2L)
    launch_gr_powers(st, s.aux + 128, p.nhi, p.Thi);
    // rows h L + e_lo (h >= 1) = r^(2 L h) r^(2 e_lo): one grouped product, matrix h - 1 for
    // the rows (h - 1) L .. h L - 1 of the block, each reading row e_lo of the first block
    launch_gr_mulmat_batch(st, p.nhi - 1, p.Thi + 64, 64, p.Mhi);
    bool done = false;
    if (ctx->gemm_path == MPC_GEMM_LIMB_TC) {
      GrMMArgs g = grargs(ctx);
      g.R = (p.nhi - 1) * p.L;
      g.p0 = p.Rtab;
      g.in = GrRowMap{p.L, 64, 0};
      g.Mmat = p.Mhi;
      g.mrows = p.L;
      g.out = p.Rtab + p.L * 64;
      g.om = GrRowMap{0, 64, 0};
      g_launches += 1;
      Phase kp(ctx, MPC_PROF_K_GR_MATMUL, (double)g.R * 4096);
      done = gr_matmul_tc_ex(st, g, ctx->status, ST_TIMEOUT) == 0;
      if (!done) g_launches -= 1;
    }
    for (long long h = 1; h < p.nhi && !done; ++h)
      if ((rc = gr_matmul(ctx, p.L, p.Rtab, nullptr, 1, 64, p.Mhi + (h - 1) * 4096, nullptr, 0,
                          p.Rtab + h * p.L * 64, 64)))
        return rc;
  }
  CK(cudaMemsetAsync(p.Zpq, 0, 12 * 64 * 8, st));
  // sum_e r^(2e) p_c[e], sum_e r^(2e) q_c[e]: (12 x E) . (E x 64)
  if (p.compact) {
    // Zhi[c nhi + h] = sum_{e_lo} pq_c[h L + e_lo] r^(2 e_lo) (E = nhi L: one strided view)
    GemmTerm T;
    T.A = op(pq, p.L);
    T.B = op(p.Rtab, 64);
    if ((rc = dense_gemm(ctx, 12 * p.nhi, 64, p.L, T, epi_store(p.Zhi, 64), tcs))) return rc;
    launch_gather_rows_affine(st, 12 * p.nhi, p.Thi, 1, 1, p.nhi, p.Zrep);   // T_hi[h]
    launch_gr_mul_rows(st, 12 * p.nhi, p.Zhi, p.Zrep, p.Zprod);
    launch_block_rowsum(st, 12, p.nhi, p.Zprod, p.Zpq);
  } else {
    launch_scalar_gr_sum(st, E, pq, E, 12, p.Rtab, p.Zpq);
  }
  u64* z0 = p.zt + 384;
  for (int c = 0; c < 6; ++c)   // z_c = sum r^(2e) p_c + r sum r^(2e) q_c
    launch_gr_lincomb(st, ctx->cst + CST_ONE, p.Zpq + c * 64, s.r, p.Zpq + (6 + c) * 64,
                      z0 + c * 64);
  delete phase;
  phase = new Phase(ctx, MPC_PROF_TRUNC_S);
  {  // S_{j,j'} = sum_e r^(2e) b1_{e,j} b2_{e,j'} (P0), with r^(2e) = r^(2 L e_hi) r^(2 e_lo):
     // tensor cores for the inner sums over e_lo, then sum_{e_hi} T_hi (x) S_hi as a GEMM + fold
    launch_trunc_limb_table(st, p.Rtab, p.L, p.TL8);
    launch_trunc_bit_transpose(st, p.b1, p.Epad, p.B1T);
    launch_trunc_bit_transpose(st, p.b2, p.Epad, p.B2T);
    {
      Phase kphase(ctx, MPC_PROF_K_TRUNC_S, 4096.0 * 64 * E);
      g_launches += 1;
      if (launch_trunc_s_tc(st, p.B1T, p.B2T, p.Epad, p.TL8, p.L, p.nhi, p.S_hi, ctx->status,
                            ST_TIMEOUT))
        return fail(ctx, MPC_ERR_CUDA, "verify_matmul: tensor map of the limb table");
    }
    GemmTerm T;
    // A[a][e_hi] = coefficient a of r^(2 L e_hi)
    T.A = p.compact ? op(p.Thi, 64, 1) : op(p.Rtab, p.L * 64, 1);
    T.B = op(p.S_hi, 262144);            // B[e_hi][(p, b)]
    if ((rc = dense_gemm(ctx, 64, 262144, p.nhi, T, epi_store(p.Pst, 262144),
                         p.tc_combine ? tcs : nullptr)))
      return rc;
    launch_fold_reduce_strided(st, p.Pst, 262144, 4096, p.S);
  }
  delete phase;
  phase = new Phase(ctx, MPC_PROF_TRUNC_ROUNDS);
  const u64* z = z0;
  u64* zbuf[2] = {s.z[0], s.z[1]};
  int zi = 0;
  for (int k = 1; k <= p.kd; ++k) {   // rounds folding the 64 bits of each output
    const u64 obj = make_obj(verify_id, batch, (u32)k);
    CK(cudaMemsetAsync(p.hsum, 0, 128 * 8, st));
    launch_trunc_round_h(st, p.V, p.W, p.S, k, ctx->cst + CST_LAM, p.hsum);
    CK(cudaMemsetAsync(p.S3, 0, 2 * 192 * 8, st));
    CK(cudaMemcpyAsync(p.S3, p.hsum, 512, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(p.S3 + 192, p.hsum + 64, 512, cudaMemcpyDeviceToDevice, st));
    inner_finish(ctx, p.S3, P_VER_H0, obj, s.h0);
    inner_finish(ctx, p.S3 + 192, P_VER_H2, obj, s.h2);
    reveal(ctx, P_VER_ZETA, obj, s.tmp6, s.zp);
    launch_gr_lagrange(st, s.zp, ctx->reduce_mode, ctx->cst + CST_INV, s.coef);
    launch_gr_combine_z(st, s.coef, s.h0, s.h2, z, zbuf[zi]);
    z = zbuf[zi];
    zi ^= 1;
    launch_trunc_update_vw(st, p.V, p.W, k, s.coef);
    trace_round(ctx, tr, k, s);
  }
  delete phase;
  phase = new Phase(ctx, MPC_PROF_TRUNC_MATERIALIZE);
  // materialise the folded vectors: x.[r]_1 at P0 and P1, y.[r]_2 at P0 and P2
  Vec& tx = p.dt.x[0];
  Vec& ty = p.dt.y[0];
  if (ctx->gemm_path == MPC_GEMM_LIMB_TC && p.kd == 6) {
    // one folded element per output e: -sum_j V_j b_{e,j} as a product of the bit matrix with
    // -V on the tensor cores, then (x only) the GR product with r^(2e), for each party's copy
    u64* nV = s.MM;
    u64* nW = s.MM + 4096;
    launch_neg_copy(st, p.V, 4096, nV);
    launch_neg_copy(st, p.W, 4096, nW);
    const u64* bits[4] = {p.b1, p.b1, p.b2, p.b2};
    const u64* mats[4] = {nV, nV, nW, nW};
    u64* outs[4] = {tx.c[0], tx.c[3], ty.c[1], ty.c[5]};
    auto grmm = [&](const GrMMArgs& g, double work) {
      g_launches += 1;
      Phase kp(ctx, MPC_PROF_K_GR_MATMUL, work);
      return gr_matmul_tc_ex(st, g, ctx->status, ST_TIMEOUT);
    };
    if (p.Lm) {
      // x_e = r^(2 Lm e_hi) (sum_j b_{e,j} r^(2 e_lo) (-V_j)): the per-row factor r^(2e) split
      // into two grouped GR matrix products on the tensor cores.
      const long long Lm = p.Lm, nhm = p.nhm, nB = (E + Lm - 1) / Lm;
      launch_gr_mulmat_batch(st, 64, nV, 64, p.Vm);
      if (p.compact) {   // r^(2 Lm e_hi) = T_hi[e / L] r^(2 (e mod L)), e = e_hi Lm
        u64* ra = p.Prow;
        u64* rb = p.Prow + nB * 64;
        u64* rr = p.Prow + 2 * nB * 64;
        launch_gather_rows_affine(st, nB, p.Thi, Lm, p.L, 0, ra);
        launch_gather_rows_affine(st, nB, p.Rtab, Lm, 1, p.L, rb);
        launch_gr_mul_rows(st, nB, ra, rb, rr);
        launch_gr_mulmat_batch(st, nB, rr, 64, p.Bm);
      } else {
        launch_gr_mulmat_batch(st, nB, p.Rtab, Lm * 64, p.Bm);
      }
      launch_word_transpose(st, nhm, Lm, E, p.b1, p.bT);
      GrMMArgs g = grargs(ctx);
      // Tm: rows sigma = j Lm + e_lo read r^(2 e_lo) and use matrix j; written at [e_lo][j]
      g.R = 64 * Lm;
      g.p0 = p.Rtab;
      g.in = GrRowMap{Lm, 64, 0};
      g.Mmat = p.Vm;
      g.mrows = Lm;
      g.out = p.Tm;
      g.om = GrRowMap{Lm, 4096, 64};
      if (grmm(g, 64.0 * Lm * 4096)) return fail(ctx, MPC_ERR_CUDA, "verify_matmul: r^(2e) V table");
      for (int v = 0; v < 2; ++v) {
        // rows rho = e_lo nhm + e_hi (bits b_e), matrix Tm[e_lo], result at row e
        GrMMArgs ga = grargs(ctx);
        ga.R = nhm * Lm;
        ga.p0 = p.bT;
        ga.in = GrRowMap{0, 1, 0};
        ga.a_bits = 1;
        ga.Mmat = p.Tm;
        ga.mrows = nhm;
        ga.out = outs[v];
        ga.om = GrRowMap{nhm, Lm * 64, 64};
        ga.out_lim = E * 64;
        if (grmm(ga, (double)nhm * Lm * 4096 * 8.0 / 36.0))
          return fail(ctx, MPC_ERR_CUDA, "verify_matmul: folded-vector product");
        // in place: rows e, matrix M(r^(2 Lm e_hi)) for e_hi = e / Lm
        GrMMArgs gb = grargs(ctx);
        gb.R = E;
        gb.p0 = outs[v];
        gb.in = GrRowMap{0, 64, 0};
        gb.Mmat = p.Bm;
        gb.mrows = Lm;
        gb.out = outs[v];
        gb.om = GrRowMap{0, 64, 0};
        if (grmm(gb, (double)E * 4096))
          return fail(ctx, MPC_ERR_CUDA, "verify_matmul: r^(2e) factor");
      }
    }
    for (int v = p.Lm ? 2 : 0; v < 4; ++v) {
      GrMMArgs g = grargs(ctx);
      g.R = E;
      g.p0 = bits[v];
      g.in = GrRowMap{0, 1, 0};
      g.a_bits = 1;
      g.Mmat = mats[v];
      g.out = outs[v];
      g.om = GrRowMap{0, 64, 0};
      // A has digit plane 0 only: 8 of the 36 digit-pair products (work in 36-pair units)
      if (grmm(g, (double)E * 4096 * 8.0 / 36.0))
        return fail(ctx, MPC_ERR_CUDA, "verify_matmul: folded-vector product");
      if (v < 2) {
        Phase kp(ctx, MPC_PROF_K_GR_MUL_ROWS, (double)E * 4096);
        launch_gr_mul_rows(st, E, outs[v], p.Rtab, outs[v]);
      }
    }
  } else {
    launch_trunc_materialize(st, E, p.b1, p.V, p.Rtab, p.kd, tx.c[0]);
    launch_trunc_materialize(st, E, p.b1, p.V, p.Rtab, p.kd, tx.c[3]);
    launch_trunc_materialize(st, E, p.b2, p.W, nullptr, p.kd, ty.c[1]);
    launch_trunc_materialize(st, E, p.b2, p.W, nullptr, p.kd, ty.c[5]);
  }
  delete phase;
  if ((rc = cuda_check(ctx, "trunc batch"))) return rc;
  phase = new Phase(ctx, MPC_PROF_TRUNC_TAIL);
  // the claim entering the dense rounds must not alias their round scratch
  CK(cudaMemcpyAsync(s.zinit, z, 384 * 8, cudaMemcpyDeviceToDevice, st));
  p.dt.cur = 0;
  rc = run_dense(ctx, verify_id, batch, p.dt, p.Dt, s.zinit, p.kd + 1, p.R1, s, p.ivt, tr);
  delete phase;
  return rc;
}

// workspace of a standalone truncation (mpc_trunc)
struct TruncCallPlan {
  u64* rx;   // 6n: the pairs' r_x shares in the mask components
  u64 *gp2, *gq2, *gp2i, *gq2i, *mp1, *mq1, *mpi1, *mqi1, *mpi2, *mqi2;   // pair messages
  u64 *d1, *d2, *d1p0, *d2p0, *d1_at_p2, *d2_at_p1;                      // mask switch
  u32* hs[4];
  u32* dg;   // 4 x 8 digest words
};

TruncCallPlan plan_trunc_call(Arena& a, long long n) {
  TruncCallPlan p;
  p.rx = a.take<u64>(6 * n);
  u64** bufs[] = {&p.gp2, &p.gq2, &p.gp2i, &p.gq2i, &p.mp1, &p.mq1, &p.mpi1, &p.mqi1, &p.mpi2,
                  &p.mqi2, &p.d1, &p.d2, &p.d1p0, &p.d2p0, &p.d1_at_p2, &p.d2_at_p1};
  for (u64** b : bufs) *b = a.take<u64>(n);
  for (int i = 0; i < 4; ++i) p.hs[i] = a.take<u32>((long long)hash_scratch_words(n));
  p.dg = a.take<u32>(32);
  return p;
}

// Every chunk of a truncation batch (batches 1, 2, ... of verify_id); trace: chunk after chunk.
int verify_trunc_batch(mpc_ctx* ctx, TruncBatch& b, const Small& s, void* tcs, const u64* pq,
                       int trunc_bits, u64 verify_id, u64 call_id, u64* tr, const u64* row_keys,
                       long long N) {
  for (long long i = 0; i < b.nchunks; ++i) {
    TruncPlan& tp = b.tp[i == b.nchunks - 1 ? 1 : 0];
    const int rc = verify_trunc_chunk(ctx, tp, s, tcs, pq, b.E, i * b.C, trunc_bits, verify_id,
                                      (u32)(1 + i), call_id, tr, row_keys, N);
    if (rc) return rc;
    if (tr) tr += (long long)(tp.R1 + 1) * TRACE_ROUND;
  }
  return MPC_OK;
}

}  // namespace

// =================================================================================================
// C-ABI
// =================================================================================================
extern "C" {

int mpc_create(const mpc_config* cfg, mpc_ctx** out) {
  if (!out) return MPC_ERR_ARG;
  *out = nullptr;
  if (!cfg) return MPC_ERR_ARG;
  if (cfg->reduce_mode != MPC_REDUCE_POINT_X && cfg->reduce_mode != MPC_REDUCE_POINT_2)
    return MPC_ERR_ARG;
  if (cfg->gemm_path != MPC_GEMM_U64 && cfg->gemm_path != MPC_GEMM_LIMB_TC) return MPC_ERR_ARG;
  mpc_ctx* ctx = new mpc_ctx();
  ctx->device = cfg->device;
  ctx->reduce_mode = cfg->reduce_mode;
  ctx->gemm_path = cfg->gemm_path;
  auto bail = [&](const char* what, cudaError_t e) {
    std::fprintf(stderr, "mpc_create: %s: %s\n", what, cudaGetErrorString(e));
    if (ctx->cst) cudaFree(ctx->cst);
    if (ctx->own_stream && ctx->st) cudaStreamDestroy(ctx->st);
    delete ctx;
    return MPC_ERR_CUDA;
  };
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return bail("cudaSetDevice", e);
  if (cfg->stream) {
    ctx->st = (cudaStream_t)cfg->stream;
  } else {
    e = cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail("cudaStreamCreate", e);
    ctx->own_stream = true;
  }
  // constants block + status word + key staging
  e = cudaMalloc(&ctx->cst, CST_WORDS * 8 + 256 + 256);
  if (e != cudaSuccess) return bail("cudaMalloc", e);
  ctx->status = reinterpret_cast<u32*>(reinterpret_cast<char*>(ctx->cst) + CST_WORDS * 8);
  u32* keys_dev = reinterpret_cast<u32*>(reinterpret_cast<char*>(ctx->cst) + CST_WORDS * 8 + 256);
  Key master;
  std::memcpy(master.k, cfg->seed, 32);
  k_derive_keys<<<1, 32, 0, ctx->st>>>(master, keys_dev);
  launch_gr_inverses(ctx->st, ctx->cst + CST_INV);
  launch_mode_consts(ctx->st, ctx->reduce_mode, ctx->cst + CST_LAM);
  k_init_consts<<<1, 64, 0, ctx->st>>>(ctx->reduce_mode, ctx->cst);
  e = cudaMemsetAsync(ctx->status, 0, sizeof(u32), ctx->st);
  if (e != cudaSuccess) return bail("cudaMemset", e);
  u32 kh[24];
  e = cudaMemcpyAsync(kh, keys_dev, sizeof(kh), cudaMemcpyDeviceToHost, ctx->st);
  if (e != cudaSuccess) return bail("key copy", e);
  e = cudaStreamSynchronize(ctx->st);
  if (e != cudaSuccess) return bail("init", e);
  std::memcpy(ctx->k01.k, kh, 32);
  std::memcpy(ctx->k02.k, kh + 8, 32);
  std::memcpy(ctx->k12.k, kh + 16, 32);
  *out = ctx;
  return MPC_OK;
}

void mpc_destroy(mpc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  if (ctx->copy_st) {
    cudaStreamSynchronize(ctx->copy_st);
    cudaStreamDestroy(ctx->copy_st);
  }
  for (cudaEvent_t e : ctx->copy_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->order_ev) cudaEventDestroy(ctx->order_ev);
  for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
  if (ctx->cst) cudaFree(ctx->cst);
  if (ctx->own_stream && ctx->st) cudaStreamDestroy(ctx->st);
  delete ctx;
}

const char* mpc_last_error(const mpc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int mpc_h2d_async(mpc_ctx* ctx, void* dst, const void* src, size_t bytes, int slot) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (!dst || !src || bytes == 0 || slot < 0 || slot >= MPC_H2D_SLOTS)
    return fail(ctx, MPC_ERR_ARG, "h2d_async: bad argument");
  if (!ctx->copy_st) CK(cudaStreamCreateWithFlags(&ctx->copy_st, cudaStreamNonBlocking));
  if (!ctx->copy_ev[slot]) CK(cudaEventCreateWithFlags(&ctx->copy_ev[slot], cudaEventDisableTiming));
  if (!ctx->order_ev) CK(cudaEventCreateWithFlags(&ctx->order_ev, cudaEventDisableTiming));
  CK(cudaEventRecord(ctx->order_ev, ctx->st));   // after the work that may still read dst
  CK(cudaStreamWaitEvent(ctx->copy_st, ctx->order_ev, 0));
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->copy_st));
  CK(cudaEventRecord(ctx->copy_ev[slot], ctx->copy_st));
  return MPC_OK;
}

int mpc_d2h_async(mpc_ctx* ctx, void* dst, const void* src, size_t bytes, int slot) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (!dst || !src || bytes == 0 || slot < 0 || slot >= MPC_H2D_SLOTS)
    return fail(ctx, MPC_ERR_ARG, "d2h_async: bad argument");
  if (!ctx->copy_st) CK(cudaStreamCreateWithFlags(&ctx->copy_st, cudaStreamNonBlocking));
  if (!ctx->copy_ev[slot]) CK(cudaEventCreateWithFlags(&ctx->copy_ev[slot], cudaEventDisableTiming));
  if (!ctx->order_ev) CK(cudaEventCreateWithFlags(&ctx->order_ev, cudaEventDisableTiming));
  CK(cudaEventRecord(ctx->order_ev, ctx->st));   // after the work that writes src
  CK(cudaStreamWaitEvent(ctx->copy_st, ctx->order_ev, 0));
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->copy_st));
  CK(cudaEventRecord(ctx->copy_ev[slot], ctx->copy_st));
  return MPC_OK;
}

int mpc_h2d_wait(mpc_ctx* ctx, int slot) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (slot < 0 || slot >= MPC_H2D_SLOTS) return fail(ctx, MPC_ERR_ARG, "h2d_wait: bad slot");
  if (!ctx->copy_ev[slot]) return MPC_OK;   // nothing was issued under this slot
  CK(cudaStreamWaitEvent(ctx->st, ctx->copy_ev[slot], 0));
  return MPC_OK;
}

int mpc_set_stream(mpc_ctx* ctx, void* stream) {
  if (!ctx || !stream) return MPC_ERR_ARG;
  if (ctx->own_stream && ctx->st) {
    cudaStreamSynchronize(ctx->st);
    cudaStreamDestroy(ctx->st);
    ctx->own_stream = false;
  }
  ctx->st = (cudaStream_t)stream;
  return MPC_OK;
}

int mpc_sync(mpc_ctx* ctx) {
  if (!ctx) return MPC_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->st));
  u32 stv = 0;
  return read_status(ctx, &stv);
}

int mpc_status(const mpc_ctx* ctx) {
  if (!ctx) return MPC_ERR_ARG;
  return ctx->aborted ? MPC_ERR_ABORT : MPC_OK;
}

int mpc_set_tuning(mpc_ctx* ctx, const mpc_tuning* tune) {
  if (!ctx) return MPC_ERR_ARG;
  mpc_tuning t = default_tuning();
  if (tune) {
    if (tune->trunc_block < 0 || tune->trunc_chunk < 0 || tune->row_split < 0 ||
        tune->tc_combine_min < 0 || tune->gemm_split_min < 0 || tune->gram_split < 0 ||
        tune->fold_batch_max < 0 || tune->trunc_block % 128 || tune->row_split % 128 ||
        tune->trunc_block > 65536 || tune->gram_split > 65535 || tune->gr_producers < 0 ||
        tune->gr_producers > 3 || (tune->gr_drain_warps != 0 && tune->gr_drain_warps != 8 &&
                                   tune->gr_drain_warps != 16))
      return fail(ctx, MPC_ERR_ARG, "set_tuning: value out of range");
    if (tune->trunc_block) t.trunc_block = tune->trunc_block;
    if (tune->trunc_chunk) t.trunc_chunk = tune->trunc_chunk;
    t.row_split = tune->row_split;
    if (tune->tc_combine_min) t.tc_combine_min = tune->tc_combine_min;
    if (tune->gemm_split_min) t.gemm_split_min = tune->gemm_split_min;
    if (tune->gram_split) t.gram_split = tune->gram_split;
    if (tune->fold_batch_max) t.fold_batch_max = tune->fold_batch_max;
    if (tune->gr_producers) t.gr_producers = tune->gr_producers;
    if (tune->gr_drain_warps) t.gr_drain_warps = tune->gr_drain_warps;
  }
  ctx->tune = t;
  return MPC_OK;
}

int mpc_get_tuning(const mpc_ctx* ctx, mpc_tuning* out) {
  if (!ctx || !out) return MPC_ERR_ARG;
  *out = ctx->tune;
  return MPC_OK;
}

int64_t mpc_trace_words(const mpc_ctx* ctx, int op, int64_t a, int64_t b, int64_t c,
                        int trunc_bits, int R_main, int R_trunc) {
  switch (op) {
    case MPC_OP_VERIFY_MULT:
    case MPC_OP_VERIFY_MULT_CALLS:
      if (a <= 0) return -1;
      return (int64_t)((R_main < 0 ? default_R(a) : R_main) + 1) * TRACE_ROUND;
    case MPC_OP_VERIFY_MATMUL: {
      if (a <= 0 || b <= 0 || c <= 0 || trunc_bits > 63) return -1;
      int64_t w = (int64_t)((R_main < 0 ? default_R(c) : R_main) + 1) * TRACE_ROUND;
      if (trunc_bits >= 0) {
        const mpc_tuning tu = ctx ? ctx->tune : default_tuning();
        long long n = 0, C = 0;
        trunc_chunks(a * b, tu, &n, &C);
        if (n > MAX_TRUNC_CHUNKS) return -1;
        for (long long i = 0; i < n; ++i) {
          const long long Ei = i == n - 1 ? a * b - (n - 1) * C : C;
          w += (int64_t)((R_trunc < 0 ? default_R(64 * Ei) : R_trunc) + 1) * TRACE_ROUND;
        }
      }
      return w;
    }
    case MPC_OP_VERIFY_TRUNC: {
      if (a <= 0) return -1;
      const mpc_tuning tu = ctx ? ctx->tune : default_tuning();
      long long n = 0, C = 0;
      trunc_chunks(a, tu, &n, &C);
      if (n > MAX_TRUNC_CHUNKS) return -1;
      int64_t w = 0;
      for (long long i = 0; i < n; ++i) {
        const long long Ei = i == n - 1 ? a - (n - 1) * C : C;
        w += (int64_t)((R_trunc < 0 ? default_R(64 * Ei) : R_trunc) + 1) * TRACE_ROUND;
      }
      return w;
    }
    default:
      return -1;
  }
}

namespace {
void nl_plan_take(Arena& a, int nst, const long long np[2]);   // workspace of a non-linear layer
}

int64_t mpc_workspace_size(const mpc_ctx* ctx, int op, int64_t a, int64_t b, int64_t c,
                           int trunc_bits, int R_main, int R_trunc) {
  (void)ctx;
  Arena ar{nullptr, 0, 0, true};
  switch (op) {
    case MPC_OP_SHARE:
      if (a < 0) return -1;
      ar.take<u64>(a);
      ar.take<u64>(a);
      break;
    case MPC_OP_MULT:
      if (a < 0) return -1;
      for (int i = 0; i < 6; ++i) ar.take<u64>(a);
      break;
    case MPC_OP_MATMUL:
      if (a <= 0 || b <= 0 || c <= 0) return -1;
      plan_matmul(ar, a, b, c, trunc_bits >= 0, ctx && ctx->gemm_path == MPC_GEMM_LIMB_TC);
      break;
    case MPC_OP_VERIFY_MULT:
      if (a <= 0) return -1;
      plan_vmult(ar, a, R_main);
      break;
    case MPC_OP_VERIFY_MULT_CALLS:
      if (a <= 0) return -1;
      plan_vmult_calls(ar, a, R_main);
      break;
    case MPC_OP_VERIFY_MATMUL: {
      if (a <= 0 || b <= 0 || c <= 0 || trunc_bits > 63) return -1;
      VMatPlan vp;
      if (!plan_vmat(ar, a, b, c, trunc_bits, R_main, R_trunc,
                     ctx && ctx->gemm_path == MPC_GEMM_LIMB_TC, ctx ? ctx->tune : default_tuning(),
                     vp))
        return -1;
      break;
    }
    case MPC_OP_RELU: {
      if (a <= 0) return -1;
      const long long np[2] = {64 * ((a + 63) / 64), 0};
      nl_plan_take(ar, 1, np);
      break;
    }
    case MPC_OP_MAXPOOL2: {
      if (a <= 0 || b <= 0 || c <= 0 || (b & 1) || (c & 1)) return -1;
      const long long nw = a * (b / 2) * (c / 2);
      const long long np[2] = {64 * ((2 * nw + 63) / 64), 64 * ((nw + 63) / 64)};
      nl_plan_take(ar, 2, np);
      break;
    }
    case MPC_OP_RECONSTRUCT:
      if (a < 0) return -1;
      plan_rec(ar, a, true);
      break;
    case MPC_OP_SHARE_FIXED:
      if (a < 0) return -1;
      ar.take<u64>(a);
      ar.take<double>(a);
      ar.take<u64>(a);
      ar.take<u64>(a);
      break;
    case MPC_OP_RECONSTRUCT_FIXED:
      if (a < 0) return -1;
      ar.take<u64>(a);
      ar.take<double>(a);
      plan_rec(ar, a, false);
      break;
    case MPC_OP_TRUNC:
      if (a <= 0) return -1;
      plan_trunc_call(ar, a);
      break;
    case MPC_OP_VERIFY_TRUNC: {
      if (a <= 0) return -1;
      VTruncPlan vp;
      if (!plan_vtrunc(ar, a, R_trunc, ctx && ctx->gemm_path == MPC_GEMM_LIMB_TC,
                       ctx ? ctx->tune : default_tuning(), vp))
        return -1;
      break;
    }
    default:
      return -1;
  }
  return (int64_t)ar.off;
}

int mpc_share_input(mpc_ctx* ctx, uint64_t call_id, const uint64_t* x, int x_on_host, int64_t n,
                    uint64_t* xs, void* workspace, size_t workspace_bytes) {
  return mpc_share_input_from(ctx, call_id, 0, x, x_on_host, n, xs, workspace, workspace_bytes);
}

int mpc_share_input_from(mpc_ctx* ctx, uint64_t call_id, int owner, const uint64_t* x,
                         int x_on_host, int64_t n, uint64_t* xs, void* workspace,
                         size_t workspace_bytes) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (n < 0) return fail(ctx, MPC_ERR_SHAPE, "n < 0");
  if (owner < 0 || owner > 2) return fail(ctx, MPC_ERR_ARG, "share_input: owner must be 0, 1 or 2");
  if (n == 0) return MPC_OK;
  if (!x || !xs || !id_ok(call_id)) return fail(ctx, MPC_ERR_ARG, "share_input: bad argument");
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  u64* stage = ar.take<u64>(n);
  u64* mout = ar.take<u64>(n);
  if (!workspace || !ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "share_input: workspace too small");
  Phase phase(ctx, MPC_PROF_SHARE);
  const u64* xd = (const u64*)x;
  if (x_on_host) {
    CK(cudaMemcpyAsync(stage, x, (size_t)n * 8, cudaMemcpyHostToDevice, ctx->st));
    xd = stage;
  }
  launch_share_input(ctx->st, xd, n, ctx->k01, ctx->k02, make_obj(call_id, 0, 0), (u64*)xs, mout);
  // m_x: components 2 (P1) and 4 (P2).  The owner P0 sends it to both; P1 or P2 keeps its own
  // copy and sends one message to the other.  A message arriving at P1 is fault site MX_COPY_P1.
  u64* m1 = (u64*)xs + 2 * n;
  u64* m2 = (u64*)xs + 4 * n;
  if (owner == 1)
    CK(cudaMemcpyAsync(m1, mout, (size_t)n * 8, cudaMemcpyDeviceToDevice, ctx->st));
  else if ((rc = deliver(ctx, MPC_PHASE_ONLINE, MPC_PROTO_SHARE, mout, m1, n, MPC_SITE_MX_COPY_P1)))
    return rc;
  if (owner == 2)
    CK(cudaMemcpyAsync(m2, mout, (size_t)n * 8, cudaMemcpyDeviceToDevice, ctx->st));
  else if ((rc = deliver(ctx, MPC_PHASE_ONLINE, MPC_PROTO_SHARE, mout, m2, n, -1)))
    return rc;
  return cuda_check(ctx, "share_input");
}

int mpc_mult(mpc_ctx* ctx, uint64_t call_id, const uint64_t* xs, const uint64_t* ys, int64_t n,
             uint64_t* zs, void* workspace, size_t workspace_bytes) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (n <= 0) return fail(ctx, MPC_ERR_SHAPE, "mult: n <= 0");
  if (!xs || !ys || !zs || !id_ok(call_id)) return fail(ctx, MPC_ERR_ARG, "mult: bad argument");
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  u64* g2o = ar.take<u64>(n);
  u64* g2i = ar.take<u64>(n);
  u64* p1o = ar.take<u64>(n);
  u64* p2o = ar.take<u64>(n);
  u64* p1i = ar.take<u64>(n);
  u64* p2i = ar.take<u64>(n);
  if (!workspace || !ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "mult: workspace too small");
  Phase phase(ctx, MPC_PROF_MULT);
  const u64 obj = make_obj(call_id, 0, 0);
  launch_mult_offline(ctx->st, xs, ys, n, ctx->k01, ctx->k02, obj, zs, g2o);
  if ((rc = deliver(ctx, MPC_PHASE_OFFLINE, MPC_PROTO_MULT, g2o, g2i, n, MPC_SITE_GAMMA2))) return rc;
  launch_mult_online(ctx->st, xs, ys, n, ctx->k01, obj, g2i, p1o, p2o);
  if ((rc = deliver(ctx, MPC_PHASE_ONLINE, MPC_PROTO_MULT, p1o, p2i, n, MPC_SITE_MZ1))) return rc;
  if ((rc = deliver(ctx, MPC_PHASE_ONLINE, MPC_PROTO_MULT, p2o, p1i, n, MPC_SITE_MZ2))) return rc;
  launch_exchange_finish(ctx->st, n, p1o, p1i, p2o, p2i, zs, -1, nullptr);
  ctx->pending.insert((call_id << 1) | 0);
  return cuda_check(ctx, "mult");
}

int mpc_matmul(mpc_ctx* ctx, uint64_t call_id, const uint64_t* xs, const uint64_t* ws_,
               int64_t M, int64_t N, int64_t K, int trunc_bits, uint64_t* zpre, uint64_t* zout,
               uint64_t* pq, void* workspace, size_t workspace_bytes) {
  return mpc_matmul_keyed(ctx, call_id, xs, ws_, M, N, K, trunc_bits, nullptr, zpre, zout, pq,
                          workspace, workspace_bytes);
}

int mpc_matmul_keyed(mpc_ctx* ctx, uint64_t call_id, const uint64_t* xs, const uint64_t* ws_,
                     int64_t M, int64_t N, int64_t K, int trunc_bits, const uint64_t* row_keys,
                     uint64_t* zpre, uint64_t* zout, uint64_t* pq, void* workspace,
                     size_t workspace_bytes) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (M <= 0 || N <= 0 || K <= 0) return fail(ctx, MPC_ERR_SHAPE, "matmul: bad shape");
  if (trunc_bits > 63) return fail(ctx, MPC_ERR_ARG, "matmul: trunc_bits > 63");
  const bool trunc = trunc_bits >= 0;
  if (!xs || !ws_ || !zpre || !id_ok(call_id) || (trunc && (!zout || !pq || zout == zpre)))
    return fail(ctx, MPC_ERR_ARG, "matmul: bad argument");
  const long long E = M * N;
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  const bool tc = ctx->gemm_path == MPC_GEMM_LIMB_TC;
  MatmulPlan p = plan_matmul(ar, M, N, K, trunc, tc);
  // the parties' local products: CUDA-core u64 GEMM or the limb-split tensor-core GEMM
  auto party_gemm = [&](int nterms, const GemmTerm* T, const Epi& e) -> int {
    if (!tc) {
      gemm_u64(ctx->st, M, N, K, nterms, T, e, 1);
      return MPC_OK;
    }
    g_launches += 4;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ctx->prof) {
      e0 = prof_event(ctx);
      e1 = prof_event(ctx);
      ctx->recs.push_back({MPC_PROF_K_LIMB_GEMM, e0, e1, (double)M * N * K * nterms});
    }
    const int r = limb_gemm_tc(ctx->st, M, N, K, nterms, T, e, p.tc, ctx->status, ST_TIMEOUT, e0, e1,
                               ctx->tune.gemm_split_min);
    return r ? fail(ctx, MPC_ERR_CUDA, "matmul: tensor-core GEMM setup failed") : MPC_OK;
  };
  if (!workspace || !ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "matmul: workspace too small");
  cudaStream_t st = ctx->st;
  const u64 obj = make_obj(call_id, 0, 0);
  const u64 M1 = ~0ull;
  if (trunc) {   // Pi_Trunc preprocessing first: it assigns the product wire's mask
    Phase phase(ctx, MPC_PROF_TRUNC_PAIRS);
    launch_trunc_p0(st, E, ctx->k01, ctx->k02, obj, trunc_bits, zpre, zout, pq, p.gp2, p.gq2,
                    p.mp1, p.mq1, (const u64*)row_keys, N);
    const int ph = MPC_PHASE_OFFLINE, pr = MPC_PROTO_TRUNC;
    if ((rc = deliver(ctx, ph, pr, p.gp2, p.gp2i, E, MPC_SITE_GAMMA2))) return rc;
    if ((rc = deliver(ctx, ph, pr, p.mp1, p.mpi2, E, MPC_SITE_MZ1))) return rc;
    if ((rc = deliver(ctx, ph, pr, p.gp2i, p.mpi1, E, MPC_SITE_MZ2))) return rc;
    if ((rc = deliver(ctx, ph, pr, p.gq2, p.gq2i, E, MPC_SITE_GAMMA2))) return rc;
    if ((rc = deliver(ctx, ph, pr, p.mq1, p.mqi2, E, MPC_SITE_MZ1))) return rc;
    if ((rc = deliver(ctx, ph, pr, p.gq2i, p.mqi1, E, MPC_SITE_MZ2))) return rc;
    launch_trunc_finish(st, E, ctx->k01, ctx->k02, obj, trunc_bits, p.mpi1, p.mqi1, p.mpi2,
                        p.mqi2, p.gp2i, p.gq2i, p.mp1, p.mq1, zpre, zout, pq, (const u64*)row_keys, N);
  } else {
    launch_fill_masks(st, E, ctx->k01, ctx->k02, P_INNER, obj, zpre);
  }
  const u64* X = xs;
  const u64* W = ws_;
  const long long MK = M * K, KN = K * N;
  {  // P0, offline: Gamma = (R_X1 + R_X2)(R_W1 + R_W2) + r_Z; message [Gamma]_2 = Gamma - [Gamma]_1
    Phase phase(ctx, MPC_PROF_GEMM);
    GemmTerm T;
    T.A = op(X, K, 0, X + MK, 1);
    T.B = op(W, N, 0, W + KN, 1);
    Epi e = epi_store(p.g2o, N);
    e.add0 = zpre;
    e.add1 = zpre + E;
    e.prf_sign = M1;
    e.key = ctx->k01;
    e.tag = make_tag(P_INNER, C_G1);
    e.obj = obj;
    if ((rc = party_gemm(1, &T, e))) return rc;
  }
  if ((rc = deliver(ctx, MPC_PHASE_OFFLINE, MPC_PROTO_INNER, p.g2o, p.g2i, E, MPC_SITE_GAMMA2)))
    return rc;
  {  // P1, online: [m_Z]_1 = -(M_X [R_W]_1 + [R_X]_1 M_W) + [Gamma]_1
    Phase phase(ctx, MPC_PROF_GEMM);
    GemmTerm T[2];
    T[0].A = op(X + 2 * MK, K);
    T[0].B = op(W + 3 * KN, N);
    T[1].A = op(X + 3 * MK, K);
    T[1].B = op(W + 2 * KN, N);
    Epi e = epi_store(p.mz1, N);
    e.acc_sign = M1;
    e.prf_sign = 1;
    e.key = ctx->k01;
    e.tag = make_tag(P_INNER, C_G1);
    e.obj = obj;
    if ((rc = party_gemm(2, T, e))) return rc;
  }
  {  // P2, online: [m_Z]_2 = M_X (M_W - [R_W]_2) - [R_X]_2 M_W + [Gamma]_2
    Phase phase(ctx, MPC_PROF_GEMM);
    GemmTerm T[2];
    T[0].A = op(X + 4 * MK, K);
    T[0].B = op(W + 4 * KN, N, 0, W + 5 * KN, M1);
    T[1].A = op(X + 5 * MK, K, 0, nullptr, 1, M1);
    T[1].B = op(W + 4 * KN, N);
    Epi e = epi_store(p.mz2, N);
    e.add0 = p.g2i;
    if ((rc = party_gemm(2, T, e))) return rc;
  }
  {
    Phase phase(ctx, MPC_PROF_EXCHANGE);
    if ((rc = deliver(ctx, MPC_PHASE_ONLINE, MPC_PROTO_INNER, p.mz1, p.mz1i, E, MPC_SITE_MZ1)))
      return rc;
    if ((rc = deliver(ctx, MPC_PHASE_ONLINE, MPC_PROTO_INNER, p.mz2, p.mz2i, E, MPC_SITE_MZ2)))
      return rc;
    launch_exchange_finish(st, E, p.mz1, p.mz2i, p.mz2, p.mz1i, zpre, trunc_bits,
                           trunc ? zout : nullptr);
  }
  if (!trunc && zout && zout != zpre)
    CK(cudaMemcpyAsync(zout, zpre, (size_t)E * 48, cudaMemcpyDeviceToDevice, st));
  ctx->pending.insert((call_id << 1) | 1);
  return cuda_check(ctx, "matmul");
}

namespace {
// Pi_MultVerify (Fig. PPEV) of the n triples (xs, ys, zs) in the plan's workspace, up to the
// opened Delta; the caller reads the outcome with finish_verify.
int verify_mult_body(mpc_ctx* ctx, uint64_t verify_id, const u64* xs, const u64* ys,
                     const u64* zs, long long n, VMultPlan& p, u64* trace) {
  Phase phase(ctx, MPC_PROF_VERIFY_MULT);
  cudaStream_t st = ctx->st;
  const Small& s = p.s;
  // Pi_Tran (Fig. MTP): reveal r; x'_i = r^i x_i; y lifted; z = sum r^i z_i
  reveal(ctx, P_VER_R, make_obj(verify_id, 0, 0), s.tmp6, s.r);
  int rc;
  if ((rc = power_table(ctx, s.r, p.pp, p.pw, s.aux))) return rc;
  Vec& x = p.dv.x[0];
  Vec ylift;   // y stays in ring words until the first round folds it
  for (int c = 0; c < 6; ++c) {
    launch_gr_scale_rows(st, p.pw, xs + c * n, n, x.c[c]);
    ylift.c[c] = const_cast<u64*>(ys + c * n);
  }
  CK(cudaMemsetAsync(s.zinit, 0, 384 * 8, st));
  {  // z_c = sum_i z_c[i] r^i for the 6 components at once: (6 x n) . (n x 64)
    GemmTerm T;
    T.A = op(zs, n);
    T.B = op(p.pw, 64);
    gemm_u64(st, 6, 64, n, 1, &T, epi_atomic(s.zinit, 64), nsplit_for(n));
  }
  p.dv.cur = 0;
  return run_dense(ctx, verify_id, 0, p.dv, n, s.zinit, 1, p.R, s, p.iv, trace, &ylift);
}
}  // namespace

int mpc_verify_mult(mpc_ctx* ctx, uint64_t verify_id, const uint64_t* xs, const uint64_t* ys,
                    const uint64_t* zs, int64_t n, uint64_t mult_call_id, int R,
                    void* workspace, size_t workspace_bytes, uint64_t* trace) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (n <= 0) return fail(ctx, MPC_ERR_SHAPE, "verify_mult: n <= 0");
  if (!xs || !ys || !zs || !id_ok(verify_id)) return fail(ctx, MPC_ERR_ARG, "verify_mult: bad argument");
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  VMultPlan p = plan_vmult(ar, n, R);
  if (!workspace || !ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "verify_mult: workspace too small");
  if ((rc = verify_mult_body(ctx, verify_id, xs, ys, zs, n, p, trace))) return rc;
  return finish_verify(ctx, (mult_call_id << 1) | 0);
}

int mpc_verify_mult_calls(mpc_ctx* ctx, uint64_t verify_id, int ncalls,
                          const uint64_t* const* xs, const uint64_t* const* ys,
                          const uint64_t* const* zs, const int64_t* n, const uint64_t* call_ids,
                          int R, void* workspace, size_t workspace_bytes, uint64_t* trace) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (ncalls <= 0 || !xs || !ys || !zs || !n || !call_ids || !id_ok(verify_id))
    return fail(ctx, MPC_ERR_ARG, "verify_mult_calls: bad argument");
  long long N = 0;
  for (int l = 0; l < ncalls; ++l) {
    if (n[l] <= 0 || n[l] > (1ll << 40)) return fail(ctx, MPC_ERR_SHAPE, "verify_mult_calls: bad n");
    if (!xs[l] || !ys[l] || !zs[l] || !id_ok(call_ids[l]))
      return fail(ctx, MPC_ERR_ARG, "verify_mult_calls: bad argument");
    // only products still awaiting verification, each once
    if (!ctx->pending.count((call_ids[l] << 1) | 0))
      return fail(ctx, MPC_ERR_ARG, "verify_mult_calls: a call id is not a pending mpc_mult call");
    for (int j = 0; j < l; ++j)
      if (call_ids[j] == call_ids[l])
        return fail(ctx, MPC_ERR_ARG, "verify_mult_calls: a call id is listed twice");
    N += n[l];
    if (N > (1ll << 40)) return fail(ctx, MPC_ERR_SHAPE, "verify_mult_calls: batch too large");
  }
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  VMultCallsPlan p = plan_vmult_calls(ar, N, R);
  if (!workspace || !ar.ok())
    return fail(ctx, MPC_ERR_WORKSPACE, "verify_mult_calls: workspace too small");
  // the batch: component c of call l at c N + (n[0] + ... + n[l-1]) of each gathered sharing
  long long off = 0;
  for (int l = 0; l < ncalls; ++l) {
    const size_t bytes = (size_t)n[l] * 8;
    for (int c = 0; c < 6; ++c) {
      CK(cudaMemcpyAsync(p.x + c * N + off, xs[l] + c * n[l], bytes, cudaMemcpyDeviceToDevice, ctx->st));
      CK(cudaMemcpyAsync(p.y + c * N + off, ys[l] + c * n[l], bytes, cudaMemcpyDeviceToDevice, ctx->st));
      CK(cudaMemcpyAsync(p.z + c * N + off, zs[l] + c * n[l], bytes, cudaMemcpyDeviceToDevice, ctx->st));
    }
    off += n[l];
  }
  if ((rc = verify_mult_body(ctx, verify_id, p.x, p.y, p.z, N, p.v, trace))) return rc;
  if ((rc = finish_verify(ctx, (call_ids[0] << 1) | 0))) return rc;
  for (int l = 1; l < ncalls; ++l) ctx->pending.erase((call_ids[l] << 1) | 0);
  return MPC_OK;
}

int mpc_verify_matmul(mpc_ctx* ctx, uint64_t verify_id, const uint64_t* xs, const uint64_t* ws_,
                      const uint64_t* zpre, const uint64_t* pq, int64_t M, int64_t N, int64_t K,
                      int trunc_bits, uint64_t matmul_call_id, int R_main, int R_trunc,
                      void* workspace, size_t workspace_bytes, uint64_t* trace) {
  return mpc_verify_matmul_keyed(ctx, verify_id, xs, ws_, zpre, pq, M, N, K, trunc_bits, nullptr,
                                 matmul_call_id, R_main, R_trunc, workspace, workspace_bytes,
                                 trace);
}

int mpc_verify_matmul_keyed(mpc_ctx* ctx, uint64_t verify_id, const uint64_t* xs,
                            const uint64_t* ws_, const uint64_t* zpre, const uint64_t* pq,
                            int64_t M, int64_t N, int64_t K, int trunc_bits,
                            const uint64_t* row_keys, uint64_t matmul_call_id, int R_main,
                            int R_trunc, void* workspace, size_t workspace_bytes,
                            uint64_t* trace) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (M <= 0 || N <= 0 || K <= 0) return fail(ctx, MPC_ERR_SHAPE, "verify_matmul: bad shape");
  const bool trunc = trunc_bits >= 0;
  if (!xs || !ws_ || !zpre || (trunc && !pq) || !id_ok(verify_id) || !id_ok(matmul_call_id) ||
      trunc_bits > 63)
    return fail(ctx, MPC_ERR_ARG, "verify_matmul: bad argument");
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  VMatPlan p;
  if (!plan_vmat(ar, M, N, K, trunc_bits, R_main, R_trunc, ctx->gemm_path == MPC_GEMM_LIMB_TC,
                 ctx->tune, p))
    return fail(ctx, MPC_ERR_SHAPE, "verify_matmul: more than 15 truncation chunks");
  if (!workspace || !ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "verify_matmul: workspace too small");
  cudaStream_t st = ctx->st;
  const Small& s = p.s;
  const long long MK = M * K, KN = K * N;
  // ---- batch 0: the M N inner products of Z = X W, rank-1 consolidation ----
  Phase* phase = new Phase(ctx, MPC_PROF_VERIFY_GEMM);
  reveal(ctx, P_VER_R, make_obj(verify_id, 0, 0), s.tmp6, s.r);
  launch_gr_powers(st, s.r, N, p.Q);                       // r^b
  launch_gr_mul1(st, p.Q + (N - 1) * 64, s.r, s.aux);      // rho = r^N
  launch_gr_powers(st, s.aux, M, p.P);                     // rho^a
  Vec& x = p.dv.x[0];
  Vec& y = p.dv.y[0];
  for (int c = 0; c < 6; ++c) {
    GemmTerm T;
    T.A = op(xs + c * MK, K, 1);        // Xt_k = sum_a rho^a X_ak  (K x M) . (M x 64)
    T.B = op(p.P, 64);
    if ((rc = dense_gemm(ctx, K, 64, M, T, epi_store(x.c[c], 64), p.tcs))) return rc;
    GemmTerm U;
    U.A = op(ws_ + c * KN, N);          // Wt_k = sum_b r^b W_kb   (K x N) . (N x 64)
    U.B = op(p.Q, 64);
    if ((rc = dense_gemm(ctx, K, 64, N, U, epi_store(y.c[c], 64), p.tcs))) return rc;
  }
  {  // zt = sum_a rho^a (sum_b r^b Z_ab): T = Z Q for all 6 components, then Gram with P
    GemmTerm T;
    T.A = op(zpre, N);
    T.B = op(p.Q, 64);
    if ((rc = dense_gemm(ctx, 6 * M, 64, N, T, epi_store(p.T, 64), p.tcs))) return rc;
    CK(cudaMemsetAsync(p.Pz, 0, 6 * 4096 * 8, st));
    for (int c = 0; c < 6; ++c)
      gram(ctx, p.Pz + c * 4096, p.P, nullptr, 1, 64, p.T + c * M * 64, nullptr, 1, 64, M, 1);
    launch_gr_fold_reduce(st, p.Pz, 6, s.zinit);
  }
  p.dv.cur = 0;
  rc = run_dense(ctx, verify_id, 0, p.dv, K, s.zinit, 1, p.R0, s, p.iv, trace);
  delete phase;
  if (rc) return rc;
  // ---- batch 1: the truncation pairs, chunk by chunk ----
  if (trunc &&
      (rc = verify_trunc_batch(ctx, p.tb, s, p.tcs, pq, trunc_bits, verify_id, matmul_call_id,
                               trace ? trace + (long long)(p.R0 + 1) * TRACE_ROUND : nullptr,
                               (const u64*)row_keys, N)))
    return rc;
  return finish_verify(ctx, (matmul_call_id << 1) | 1);
}

int mpc_reconstruct(mpc_ctx* ctx, const uint64_t* xs, int64_t n, uint64_t* out, int out_on_host,
                    void* workspace, size_t workspace_bytes) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (n <= 0) return fail(ctx, MPC_ERR_SHAPE, "reconstruct: n <= 0");
  if (!xs || !out) return fail(ctx, MPC_ERR_ARG, "reconstruct: bad argument");
  if (!ctx->pending.empty())
    return fail(ctx, MPC_ERR_PENDING, "reconstruct: products are not verified yet");
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  RecPlan p = plan_rec(ar, n, out_on_host != 0);
  if (!workspace || !ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "reconstruct: workspace too small");
  Phase* phase = new Phase(ctx, MPC_PROF_REC);
  cudaStream_t st = ctx->st;
  const int ph = MPC_PHASE_ONLINE, pr = MPC_PROTO_REC;
  if ((rc = deliver(ctx, ph, pr, xs, p.in_p2_r1, n, -1))) return rc;             // P0 -> P2 [r]_1
  if ((rc = deliver(ctx, ph, pr, xs + n, p.in_p1_r2, n, MPC_SITE_REC_MSG))) return rc;  // P0 -> P1
  if ((rc = deliver(ctx, ph, pr, xs + 2 * n, p.in_p0_m, n, -1))) return rc;      // P1 -> P0 m
  u32* d = p.dg;
  launch_hash_u64(st, xs + 3 * n, n, p.hs[0], d + 0);     // P1: H([r]_1) -> P2
  launch_hash_u64(st, xs + 4 * n, n, p.hs[1], d + 8);     // P2: H(m) -> P0
  launch_hash_u64(st, xs + 5 * n, n, p.hs[2], d + 16);    // P2: H([r]_2) -> P1
  count_msgs(ctx, ph, pr, 3, 32);
  launch_hash_u64(st, p.in_p2_r1, n, p.hs[3], d + 24);    // P2 hashes received [r]_1
  launch_hash_u64(st, p.in_p0_m, n, p.hs[4], d + 32);     // P0 hashes received m
  launch_hash_u64(st, p.in_p1_r2, n, p.hs[5], d + 40);    // P1 hashes received [r]_2
  launch_digest_check(st, d + 0, d + 24, d + 8, d + 32, d + 16, d + 40, ctx->status, ST_ABORT);
  u64* o = out_on_host ? p.out_dev : (u64*)out;
  launch_open_p1(st, xs + 2 * n, xs + 3 * n, p.in_p1_r2, n, o);
  if (out_on_host) CK(cudaMemcpyAsync(out, o, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
  delete phase;
  if ((rc = cuda_check(ctx, "reconstruct"))) return rc;
  u32 stv = 0;
  if ((rc = read_status(ctx, &stv))) return rc;
  if (stv & ST_ABORT) {
    ctx->aborted = true;
    if (out_on_host) std::memset(out, 0, (size_t)n * 8);
    else cudaMemsetAsync(out, 0, (size_t)n * 8, st);
    return fail(ctx, MPC_ERR_ABORT, "Pi_Rec: inconsistent messages");
  }
  return MPC_OK;
}

int mpc_ledger(const mpc_ctx* ctx, uint64_t* bytes, uint64_t* messages) {
  if (!ctx || !bytes) return MPC_ERR_ARG;
  for (int a = 0; a < MPC_NPHASE; ++a)
    for (int b = 0; b < MPC_NPROTO; ++b) bytes[a * MPC_NPROTO + b] = ctx->ledger[a][b];
  if (messages) *messages = ctx->nmsg;
  return MPC_OK;
}

void mpc_ledger_reset(mpc_ctx* ctx) {
  if (!ctx) return;
  std::memset(ctx->ledger, 0, sizeof(ctx->ledger));
  ctx->nmsg = 0;
}

int mpc_inject_fault(mpc_ctx* ctx, int site, uint64_t index, uint64_t xor_mask) {
  if (!ctx || site < 0 || site >= MPC_NSITE) return MPC_ERR_ARG;
  ctx->fault[site] = {true, index, site == MPC_SITE_HIGH_BIT ? (1ull << 63) : xor_mask};
  return MPC_OK;
}

int mpc_profile(mpc_ctx* ctx, int enable) {
  if (!ctx) return MPC_ERR_ARG;
  if (enable) {
    ctx->recs.clear();
    ctx->pool_used = 0;
  }
  ctx->prof = enable != 0;
  return MPC_OK;
}

int mpc_profile_read(mpc_ctx* ctx, double* ms, uint64_t* count, double* work) {
  if (!ctx || !ms) return MPC_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->st));
  for (int i = 0; i < MPC_NPROF; ++i) {
    ms[i] = 0.0;
    if (count) count[i] = 0;
    if (work) work[i] = 0.0;
  }
  for (const auto& r : ctx->recs) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    if (r.id >= 0 && r.id < MPC_NPROF) {
      ms[r.id] += t;
      if (count) count[r.id] += 1;
      if (work) work[r.id] += r.work;
    }
  }
  ctx->recs.clear();
  ctx->pool_used = 0;
  return MPC_OK;
}

uint64_t mpc_launch_count(void) { return g_launches; }


// ---- layer-level calls -----------------------------------------------------------------------
int mpc_share_fixed(mpc_ctx* ctx, uint64_t call_id, int owner, const double* x, int x_on_host,
                    int64_t n, int frac_bits, uint64_t* xs, void* workspace,
                    size_t workspace_bytes) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (n < 0) return fail(ctx, MPC_ERR_SHAPE, "share_fixed: n < 0");
  if (frac_bits < 0 || frac_bits > 62) return fail(ctx, MPC_ERR_ARG, "share_fixed: frac_bits");
  if (n == 0) return MPC_OK;
  if (!x || !xs || !workspace) return fail(ctx, MPC_ERR_ARG, "share_fixed: bad argument");
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  u64* enc = ar.take<u64>(n);
  double* stage = ar.take<double>(n);
  if (!ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "share_fixed: workspace too small");
  const double* xd = x;
  if (x_on_host) {
    CK(cudaMemcpyAsync(stage, x, (size_t)n * 8, cudaMemcpyHostToDevice, ctx->st));
    xd = stage;
  }
  {
    Phase phase(ctx, MPC_PROF_SHARE);
    launch_encode_fixed(ctx->st, xd, n, frac_bits, enc);
    g_launches += 1;
  }
  rc = mpc_share_input_from(ctx, call_id, owner, enc, 0, n, xs, (char*)workspace + ar.off,
                            workspace_bytes > ar.off ? workspace_bytes - ar.off : 0);
  if (rc == MPC_OK && x_on_host) CK(cudaStreamSynchronize(ctx->st));   // x may be reused
  return rc;
}

int mpc_reconstruct_fixed(mpc_ctx* ctx, const uint64_t* xs, int64_t n, int frac_bits, double* out,
                          int out_on_host, void* workspace, size_t workspace_bytes) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (n <= 0) return fail(ctx, MPC_ERR_SHAPE, "reconstruct_fixed: n <= 0");
  if (frac_bits < 0 || frac_bits > 62 || !xs || !out || !workspace)
    return fail(ctx, MPC_ERR_ARG, "reconstruct_fixed: bad argument");
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  u64* v = ar.take<u64>(n);
  double* stage = ar.take<double>(n);
  if (!ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "reconstruct_fixed: workspace too small");
  rc = mpc_reconstruct(ctx, xs, n, v, 0, (char*)workspace + ar.off,
                       workspace_bytes > ar.off ? workspace_bytes - ar.off : 0);
  if (rc) {
    if (out_on_host) std::memset(out, 0, (size_t)n * 8);
    return rc;
  }
  {
    Phase phase(ctx, MPC_PROF_REC);
    launch_decode_fixed(ctx->st, v, n, frac_bits, out_on_host ? stage : out);
    g_launches += 1;
  }
  if (out_on_host) {
    CK(cudaMemcpyAsync(out, stage, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  return cuda_check(ctx, "reconstruct_fixed");
}

int mpc_conv2d(mpc_ctx* ctx, uint64_t call_id, const uint64_t* xs, const uint64_t* ws_,
               const int32_t geom[8], int64_t C_out, int trunc_bits, const uint64_t* row_keys,
               uint64_t* cols, uint64_t* zpre, uint64_t* zout, uint64_t* pq, void* workspace,
               size_t workspace_bytes) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (!geom || !xs || !cols) return fail(ctx, MPC_ERR_ARG, "conv2d: bad argument");
  ConvGeom g;
  g.B = geom[0]; g.C = geom[1]; g.H = geom[2]; g.W = geom[3];
  g.kh = geom[4]; g.kw = geom[5]; g.stride = geom[6]; g.pad = geom[7];
  if (g.B <= 0 || g.C <= 0 || g.H <= 0 || g.W <= 0 || g.kh <= 0 || g.kw <= 0 || g.stride <= 0 ||
      g.pad < 0 || C_out <= 0)
    return fail(ctx, MPC_ERR_SHAPE, "conv2d: bad geometry");
  if (g.H + 2 * g.pad < g.kh || g.W + 2 * g.pad < g.kw)
    return fail(ctx, MPC_ERR_SHAPE, "conv2d: kernel larger than the padded image");
  g.Ho = (g.H + 2 * g.pad - g.kh) / g.stride + 1;
  g.Wo = (g.W + 2 * g.pad - g.kw) / g.stride + 1;
  launch_im2col(ctx->st, xs, g, cols);
  g_launches += 1;
  if ((rc = cuda_check(ctx, "conv2d: im2col"))) return rc;
  return mpc_matmul_keyed(ctx, call_id, cols, ws_, g.B * g.Ho * g.Wo, C_out, g.C * g.kh * g.kw,
                          trunc_bits, row_keys, zpre, zout, pq, workspace, workspace_bytes);
}

int mpc_trunc(mpc_ctx* ctx, uint64_t call_id, const uint64_t* xs, int64_t n, int t, uint64_t* out,
              uint64_t* pq, void* workspace, size_t workspace_bytes) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (n <= 0) return fail(ctx, MPC_ERR_SHAPE, "trunc: n <= 0");
  if (t < 0 || t > 63 || !xs || !out || !pq || out == xs || !id_ok(call_id))
    return fail(ctx, MPC_ERR_ARG, "trunc: bad argument");
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  TruncCallPlan p = plan_trunc_call(ar, n);
  if (!workspace || !ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "trunc: workspace too small");
  cudaStream_t st = ctx->st;
  const u64 obj = make_obj(call_id, 0, 0);
  {  // preprocessing (Fig. trunc): the pairs, as for a truncated product
    Phase phase(ctx, MPC_PROF_TRUNC_PAIRS);
    launch_trunc_p0(st, n, ctx->k01, ctx->k02, obj, t, p.rx, out, pq, p.gp2, p.gq2, p.mp1, p.mq1,
                    nullptr, n);
    const int ph = MPC_PHASE_OFFLINE, pr = MPC_PROTO_TRUNC;
    if ((rc = deliver(ctx, ph, pr, p.gp2, p.gp2i, n, MPC_SITE_GAMMA2))) return rc;
    if ((rc = deliver(ctx, ph, pr, p.mp1, p.mpi2, n, MPC_SITE_MZ1))) return rc;
    if ((rc = deliver(ctx, ph, pr, p.gp2i, p.mpi1, n, MPC_SITE_MZ2))) return rc;
    if ((rc = deliver(ctx, ph, pr, p.gq2, p.gq2i, n, MPC_SITE_GAMMA2))) return rc;
    if ((rc = deliver(ctx, ph, pr, p.mq1, p.mqi2, n, MPC_SITE_MZ1))) return rc;
    if ((rc = deliver(ctx, ph, pr, p.gq2i, p.mqi1, n, MPC_SITE_MZ2))) return rc;
    launch_trunc_finish(st, n, ctx->k01, ctx->k02, obj, t, p.mpi1, p.mqi1, p.mpi2, p.mqi2,
                        p.gp2i, p.gq2i, p.mp1, p.mq1, p.rx, out, pq, nullptr, n);
  }
  {  // online: the wire's mask switched to the pairs' r_x (checked by P0's hashes), then m >> t
    Phase phase(ctx, MPC_PROF_EXCHANGE);
    launch_trunc_remask(st, xs, p.rx, n, p.d1, p.d2, p.d1p0, p.d2p0);
    g_launches += 1;
    const int ph = MPC_PHASE_ONLINE, pr = MPC_PROTO_TRUNC;
    if ((rc = deliver(ctx, ph, pr, p.d1, p.d1_at_p2, n, MPC_SITE_TRUNC_D1))) return rc;   // P1->P2
    if ((rc = deliver(ctx, ph, pr, p.d2, p.d2_at_p1, n, -1))) return rc;                 // P2->P1
    launch_hash_u64(st, p.d1p0, n, p.hs[0], p.dg);            // P0: H(d1) -> P2
    launch_hash_u64(st, p.d2p0, n, p.hs[1], p.dg + 8);        // P0: H(d2) -> P1
    count_msgs(ctx, ph, pr, 2, 32);
    launch_hash_u64(st, p.d1_at_p2, n, p.hs[2], p.dg + 16);   // P2 hashes the d1 it received
    launch_hash_u64(st, p.d2_at_p1, n, p.hs[3], p.dg + 24);   // P1 hashes the d2 it received
    launch_digest_check(st, p.dg, p.dg + 16, p.dg + 8, p.dg + 24, p.dg, p.dg + 16, ctx->status,
                        ST_ABORT);
    launch_trunc_online(st, xs, n, p.d1, p.d2_at_p1, p.d1_at_p2, p.d2, t, out);
    g_launches += 1;
  }
  if ((rc = cuda_check(ctx, "trunc"))) return rc;
  ctx->pending.insert((call_id << 1) | 1);
  u32 stv = 0;
  if ((rc = read_status(ctx, &stv))) return rc;
  if (stv & ST_ABORT) {
    ctx->aborted = true;
    return fail(ctx, MPC_ERR_ABORT, "Pi_Trunc: a mask-switch message disagrees with P0's hash");
  }
  return MPC_OK;
}

int mpc_verify_trunc(mpc_ctx* ctx, uint64_t verify_id, const uint64_t* pq, int64_t n, int t,
                     uint64_t trunc_call_id, int R, void* workspace, size_t workspace_bytes,
                     uint64_t* trace) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (n <= 0) return fail(ctx, MPC_ERR_SHAPE, "verify_trunc: n <= 0");
  if (!pq || t < 0 || t > 63 || !id_ok(verify_id) || !id_ok(trunc_call_id))
    return fail(ctx, MPC_ERR_ARG, "verify_trunc: bad argument");
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  VTruncPlan p;
  if (!plan_vtrunc(ar, n, R, ctx->gemm_path == MPC_GEMM_LIMB_TC, ctx->tune, p))
    return fail(ctx, MPC_ERR_SHAPE, "verify_trunc: more than 15 chunks");
  if (!workspace || !ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "verify_trunc: workspace too small");
  if ((rc = verify_trunc_batch(ctx, p.tb, p.s, p.tcs, pq, t, verify_id, trunc_call_id, trace,
                               nullptr, n)))
    return rc;
  return finish_verify(ctx, (trunc_call_id << 1) | 1);
}


int mpc_test_wait_expires(mpc_ctx* ctx, int64_t cycles) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (cycles < 1 || cycles > 100000000) return fail(ctx, MPC_ERR_ARG, "test_wait_expires: cycles");
  launch_wait_expires(ctx->st, cycles, ctx->status, ST_TIMEOUT);
  g_launches += 1;
  if ((rc = cuda_check(ctx, "test_wait_expires"))) return rc;
  u32 stv = 0;
  return read_status(ctx, &stv);   // MPC_ERR_TIMEOUT, and the context is aborted
}
}  // extern "C"

// ---- accessors for other translation units of the library (not part of the C-ABI) ----------
namespace mpc3 {
namespace internal {
int ctx_guard(mpc_ctx* c) { return guard(c); }
int ctx_fail(mpc_ctx* c, int code, const char* msg) { return fail(c, code, msg); }
int ctx_deliver(mpc_ctx* c, int phase, int proto, const u64* src, u64* dst, long long n, int site) {
  return deliver(c, phase, proto, src, dst, n, site);
}
void ctx_count(mpc_ctx* c, int phase, int proto, int count, u64 bytes_each) {
  count_msgs(c, phase, proto, count, bytes_each);
}
int ctx_read_status(mpc_ctx* c, u32* out) { return read_status(c, out); }
bool ctx_has_pending(const mpc_ctx* c) { return !c->pending.empty(); }
cudaStream_t ctx_stream(const mpc_ctx* c) { return c->st; }
u32* ctx_status_word(const mpc_ctx* c) { return c->status; }
void ctx_set_aborted(mpc_ctx* c) { c->aborted = true; }
}  // namespace internal
}  // namespace mpc3

// ---- non-linear layers (Sec. 4.3) -------------------------------------------------------------
namespace {

// messages of one Pi_Mult / AND batch of up to n words
struct MsgBuf {
  u64 *g2o, *g2i, *p1o, *p2o, *p1i, *p2i;
};
MsgBuf plan_msg(Arena& a, long long n) {
  MsgBuf m;
  m.g2o = a.take<u64>(n); m.g2i = a.take<u64>(n);
  m.p1o = a.take<u64>(n); m.p2o = a.take<u64>(n);
  m.p1i = a.take<u64>(n); m.p2i = a.take<u64>(n);
  return m;
}

// A Boolean message of nw words; the AND_GAMMA2 site flips bit `index` of it (when mask & 1), the
// Boolean counterpart of an element fault; HIGH_BIT at l = 1 is the same bit flip.
int deliver_bits(mpc_ctx* ctx, int phase, int proto, const u64* src, u64* dst, long long nw, int site) {
  if (nw > 0) CK(cudaMemcpyAsync(dst, src, (size_t)nw * 8, cudaMemcpyDeviceToDevice, ctx->st));
  ctx->ledger[phase][proto] += (u64)nw * 8;
  ctx->nmsg += 1;
  if (site >= 0 && nw > 0) {
    Fault& f = ctx->fault[site];
    if (f.armed) {
      const u64 bit = f.index % (u64)(64 * nw);
      if (f.mask & 1ull) launch_xor_one(ctx->st, dst + bit / 64, 1ull << (bit % 64));
      f.armed = false;
    }
  }
  return MPC_OK;
}

// arithmetic Pi_Mult (Fig. MultP) with the streams of (purpose, obj)
int mult_p(mpc_ctx* ctx, const u64* xs, const u64* ys, long long n, u32 purpose, u64 obj, u64* zs,
           const MsgBuf& m) {
  int rc;
  launch_mult_offline_p(ctx->st, xs, ys, n, ctx->k01, ctx->k02, purpose, obj, zs, m.g2o);
  g_launches += 1;
  if ((rc = deliver(ctx, MPC_PHASE_OFFLINE, MPC_PROTO_MULT, m.g2o, m.g2i, n, MPC_SITE_GAMMA2))) return rc;
  launch_mult_online_p(ctx->st, xs, ys, n, ctx->k01, purpose, obj, m.g2i, m.p1o, m.p2o);
  g_launches += 1;
  if ((rc = deliver(ctx, MPC_PHASE_ONLINE, MPC_PROTO_MULT, m.p1o, m.p2i, n, MPC_SITE_MZ1))) return rc;
  if ((rc = deliver(ctx, MPC_PHASE_ONLINE, MPC_PROTO_MULT, m.p2o, m.p1i, n, MPC_SITE_MZ2))) return rc;
  launch_exchange_finish(ctx->st, n, m.p1o, m.p1i, m.p2o, m.p2i, zs, -1, nullptr);
  return MPC_OK;
}

// Boolean AND gates (Fig. MultP over Z_2) on nw bit-sliced words
int and_p(mpc_ctx* ctx, const u64* xs, const u64* ys, long long nw, u32 purpose, u64 obj, u64* zs,
          const MsgBuf& m) {
  int rc;
  launch_and_offline(ctx->st, xs, ys, nw, ctx->k01, ctx->k02, purpose, obj, zs, m.g2o);
  g_launches += 1;
  if ((rc = deliver_bits(ctx, MPC_PHASE_OFFLINE, MPC_PROTO_MULT, m.g2o, m.g2i, nw, MPC_SITE_AND_GAMMA2)))
    return rc;
  launch_and_online(ctx->st, xs, ys, nw, ctx->k01, purpose, obj, m.g2i, m.p1o, m.p2o);
  g_launches += 1;
  if ((rc = deliver_bits(ctx, MPC_PHASE_ONLINE, MPC_PROTO_MULT, m.p1o, m.p2i, nw, -1))) return rc;
  if ((rc = deliver_bits(ctx, MPC_PHASE_ONLINE, MPC_PROTO_MULT, m.p2o, m.p1i, nw, -1))) return rc;
  launch_xor_finish(ctx->st, nw, m.p1o, m.p1i, m.p2o, m.p2i, zs);
  g_launches += 1;
  return MPC_OK;
}

// Pi_Rec of n words inside a layer (messages, hashes, consistency check into the status word);
// P1's opening into out: m - [r]_1 - [r]_2, or m XOR [r]_1 XOR [r]_2 for a Boolean sharing.
int rec_open(mpc_ctx* ctx, const u64* xs, long long n, const RecPlan& p, u64* out, bool boolean) {
  int rc;
  cudaStream_t st = ctx->st;
  const int ph = MPC_PHASE_ONLINE, pr = MPC_PROTO_REC;
  if ((rc = deliver(ctx, ph, pr, xs, p.in_p2_r1, n, -1))) return rc;
  if ((rc = deliver(ctx, ph, pr, xs + n, p.in_p1_r2, n, boolean ? -1 : MPC_SITE_REC_MSG))) return rc;
  if ((rc = deliver(ctx, ph, pr, xs + 2 * n, p.in_p0_m, n, -1))) return rc;
  u32* d = p.dg;
  launch_hash_u64(st, xs + 3 * n, n, p.hs[0], d + 0);
  launch_hash_u64(st, xs + 4 * n, n, p.hs[1], d + 8);
  launch_hash_u64(st, xs + 5 * n, n, p.hs[2], d + 16);
  count_msgs(ctx, ph, pr, 3, 32);
  launch_hash_u64(st, p.in_p2_r1, n, p.hs[3], d + 24);
  launch_hash_u64(st, p.in_p0_m, n, p.hs[4], d + 32);
  launch_hash_u64(st, p.in_p1_r2, n, p.hs[5], d + 40);
  launch_digest_check(st, d + 0, d + 24, d + 8, d + 32, d + 16, d + 40, ctx->status, ST_ABORT);
  if (boolean) {
    launch_open_xor(st, xs + 2 * n, xs + 3 * n, p.in_p1_r2, n, out);
    g_launches += 1;
  } else {
    launch_open_p1(st, xs + 2 * n, xs + 3 * n, p.in_p1_r2, n, out);
  }
  return MPC_OK;
}

constexpr int NL_LEVELS = 6;
inline int level_planes(int l) { return l == NL_LEVELS ? 1 : 2 * (32 >> (l - 1)); }   // 64,32,..,4,1

// Buffers of one compare-select stage of np (padded) elements, W = np / 64 words per plane.
struct CSPlan {
  long long np, W;
  MsgBuf ma, mb;                 // arithmetic (64 np) and Boolean (64 W) message buffers
  u64 *b1w, *b2w, *mbw, *rbits;  // edaBit bit planes (64 W each), Boolean sharing (6 x 64 W)
  u64 *B1, *B2, *eprod, *rp;     // 6 x 64 np each
  u64 *ez, *ra, *dd;             // 6 x np: edaBit inner products, <r>, <x - r>
  u64 *delta, *dpl;              // np public words, 64 W bit planes
  u64 *G, *P, *G2, *P2;          // 6 x 64 W each
  u64 *X[NL_LEVELS + 1], *Y[NL_LEVELS + 1], *Z[NL_LEVELS + 1];   // AND triples per level
  u64 *ge, *r1w, *r2w, *r3w, *rb, *e, *dbits;                    // Boolean, W-sized
  u64 *A1, *A2, *A3, *t, *rpd, *u, *rad, *gea, *d, *prod;        // 6 x np
  RecPlan reca, recb;
  long long and_words;           // words of all AND triples (per component)
};

CSPlan plan_cs(Arena& a, long long np) {
  CSPlan p;
  p.np = np;
  p.W = np / 64;
  const long long W = p.W, N = 64 * np;
  p.ma = plan_msg(a, N);
  p.mb = plan_msg(a, 64 * W);
  p.b1w = a.take<u64>(64 * W); p.b2w = a.take<u64>(64 * W); p.mbw = a.take<u64>(64 * W);
  p.rbits = a.take<u64>(6 * 64 * W);
  p.B1 = a.take<u64>(6 * N); p.B2 = a.take<u64>(6 * N);
  p.eprod = a.take<u64>(6 * N); p.rp = a.take<u64>(6 * N);
  p.ez = a.take<u64>(6 * np); p.ra = a.take<u64>(6 * np); p.dd = a.take<u64>(6 * np);
  p.delta = a.take<u64>(np); p.dpl = a.take<u64>(64 * W);
  p.G = a.take<u64>(6 * 64 * W); p.P = a.take<u64>(6 * 64 * W);
  p.G2 = a.take<u64>(6 * 64 * W); p.P2 = a.take<u64>(6 * 64 * W);
  p.and_words = 0;
  for (int l = 1; l <= NL_LEVELS; ++l) {
    const long long nw = (long long)level_planes(l) * W;
    p.X[l] = a.take<u64>(6 * nw); p.Y[l] = a.take<u64>(6 * nw); p.Z[l] = a.take<u64>(6 * nw);
    p.and_words += nw;
  }
  p.ge = a.take<u64>(6 * W);
  p.r1w = a.take<u64>(W); p.r2w = a.take<u64>(W); p.r3w = a.take<u64>(W);
  p.rb = a.take<u64>(6 * W); p.e = a.take<u64>(6 * W); p.dbits = a.take<u64>(W);
  p.A1 = a.take<u64>(6 * np); p.A2 = a.take<u64>(6 * np); p.A3 = a.take<u64>(6 * np);
  p.t = a.take<u64>(6 * np); p.rpd = a.take<u64>(6 * np); p.u = a.take<u64>(6 * np);
  p.rad = a.take<u64>(6 * np); p.gea = a.take<u64>(6 * np); p.d = a.take<u64>(6 * np);
  p.prod = a.take<u64>(6 * np);
  p.reca = plan_rec(a, np, false);
  p.recb = plan_rec(a, W, false);
  return p;
}

// Boolean sharing (6 x nw words) whose components are the pair-known bit planes (r1, r2, m):
// P0 (r1, r2), P1 (m, r1), P2 (m, r2)
int bool_from_planes(mpc_ctx* ctx, const u64* r1, const u64* r2, const u64* m, long long nw, u64* s) {
  const u64* src[6] = {r1, r2, m, r1, m, r2};
  for (int c = 0; c < 6; ++c)
    CK(cudaMemcpyAsync(s + c * nw, src[c], (size_t)nw * 8, cudaMemcpyDeviceToDevice, ctx->st));
  return MPC_OK;
}

// <max(a, b)> into out (6 np each; out may alias neither a nor b): Sec. 4.3 compare-select
int compare_select(mpc_ctx* ctx, u64 call_id, int stage, const u64* a, const u64* b, CSPlan& p,
                   u64* out) {
  int rc;
  cudaStream_t st = ctx->st;
  const long long np = p.np, W = p.W, N = 64 * np;
  const u64 obj = make_obj(call_id, (u32)stage, 0);
  launch_addsub(st, 6 * np, a, b, 1, p.d);                                  // d = a - b
  g_launches += 1;
  // edaBits (Fig. edabits)
  launch_prf_words(st, 64 * W, ctx->k01, make_tag(P_EDABIT, C_R1), obj, p.b1w, 0ll);
  launch_prf_words(st, 64 * W, ctx->k02, make_tag(P_EDABIT, C_R2), obj, p.b2w, 0ll);
  launch_prf_words(st, 64 * W, ctx->k12, make_tag(P_EDABIT, C_M12), obj, p.mbw, 0ll);
  if ((rc = bool_from_planes(ctx, p.b1w, p.b2w, p.mbw, 64 * W, p.rbits))) return rc;
  launch_bits_to_arith(st, p.b1w, N, 0, p.B1);
  launch_bits_to_arith(st, p.b2w, N, 1, p.B2);
  g_launches += 2;
  if ((rc = mult_p(ctx, p.B1, p.B2, N, P_EDA_MULT, obj, p.eprod, p.ma))) return rc;
  launch_lin_apb_m2c(st, 6 * N, p.B1, p.B2, p.eprod, p.rp);                 // r' = b1 + b2 - 2 b1 b2
  launch_eda_inner_offline(st, np, ctx->k01, ctx->k02, obj, p.ez, p.ma.g2o);
  g_launches += 2;
  if ((rc = deliver(ctx, MPC_PHASE_OFFLINE, MPC_PROTO_INNER, p.ma.g2o, p.ma.g2i, np, MPC_SITE_GAMMA2)))
    return rc;
  launch_eda_inner_online(st, p.mbw, p.rp, np, ctx->k01, obj, p.ma.g2i, p.ma.p1o, p.ma.p2o);
  g_launches += 1;
  if ((rc = deliver(ctx, MPC_PHASE_OFFLINE, MPC_PROTO_INNER, p.ma.p1o, p.ma.p2i, np, MPC_SITE_MZ1))) return rc;
  if ((rc = deliver(ctx, MPC_PHASE_OFFLINE, MPC_PROTO_INNER, p.ma.p2o, p.ma.p1i, np, MPC_SITE_MZ2))) return rc;
  launch_exchange_finish(st, np, p.ma.p1o, p.ma.p1i, p.ma.p2o, p.ma.p2i, p.ez, -1, nullptr);
  launch_eda_compose(st, p.mbw, p.rp, p.ez, np, p.ra);
  g_launches += 2;
  // msb(d): open Delta = d - r, carry circuit over the bits of Delta + r
  launch_addsub(st, 6 * np, p.d, p.ra, 1, p.dd);
  g_launches += 1;
  if ((rc = rec_open(ctx, p.dd, np, p.reca, p.delta, false))) return rc;
  launch_trunc_bit_transpose(st, p.delta, np, p.dpl);
  launch_msb_leaves(st, p.rbits, p.dpl, W, p.G, p.P);
  g_launches += 2;
  u64 *G = p.G, *P = p.P, *G2 = p.G2, *P2 = p.P2;
  for (int l = 1; l <= NL_LEVELS; ++l) {
    const int C = 32 >> (l - 1);
    const int root = l == NL_LEVELS;
    const long long nw = (long long)level_planes(l) * W;
    launch_msb_gather(st, G, P, C, root, W, p.X[l], p.Y[l]);
    g_launches += 1;
    if ((rc = and_p(ctx, p.X[l], p.Y[l], nw, P_AND, make_obj(call_id, (u32)stage, (u32)l), p.Z[l], p.mb)))
      return rc;
    launch_msb_combine(st, G, p.Z[l], C, root, W, G2, P2);
    g_launches += 1;
    std::swap(G, G2);
    std::swap(P, P2);
  }
  launch_msb_out(st, p.rbits, G, p.dpl + 63 * W, W, 1, p.ge);               // [d >= 0] = NOT msb
  g_launches += 1;
  // daBit and B2A
  launch_prf_words(st, W, ctx->k01, make_tag(P_DABIT, C_R1), obj, p.r1w, 0ll);
  launch_prf_words(st, W, ctx->k02, make_tag(P_DABIT, C_R2), obj, p.r2w, 0ll);
  launch_prf_words(st, W, ctx->k12, make_tag(P_DABIT, C_M12), obj, p.r3w, 0ll);
  if ((rc = bool_from_planes(ctx, p.r1w, p.r2w, p.r3w, W, p.rb))) return rc;
  launch_bits_to_arith(st, p.r1w, np, 0, p.A1);
  launch_bits_to_arith(st, p.r2w, np, 1, p.A2);
  launch_bits_to_arith(st, p.r3w, np, 2, p.A3);
  g_launches += 3;
  if ((rc = mult_p(ctx, p.A1, p.A2, np, P_DA_MULT1, obj, p.t, p.ma))) return rc;
  launch_lin_apb_m2c(st, 6 * np, p.A1, p.A2, p.t, p.rpd);
  g_launches += 1;
  if ((rc = mult_p(ctx, p.rpd, p.A3, np, P_DA_MULT2, obj, p.u, p.ma))) return rc;
  launch_lin_apb_m2c(st, 6 * np, p.rpd, p.A3, p.u, p.rad);
  launch_bxor(st, 6 * W, p.ge, p.rb, p.e);
  g_launches += 2;
  if ((rc = rec_open(ctx, p.e, W, p.recb, p.dbits, true))) return rc;
  launch_b2a_apply(st, p.dbits, p.rad, np, p.gea);
  g_launches += 1;
  // out = b + (a - b) [a >= b]
  if ((rc = mult_p(ctx, p.d, p.gea, np, P_NL_MULT, obj, p.prod, p.ma))) return rc;
  launch_addsub(st, 6 * np, b, p.prod, 0, out);
  g_launches += 1;
  return cuda_check(ctx, "compare_select");
}

// ---- verification of a non-linear layer -------------------------------------------------------
struct GfPlan {   // GF(2^64) Pi_MultVerify of D AND gates
  long long D;
  int R;
  u64 *XA, *YA, *ZA;        // concatenated triples, 6 x nw words each
  u64 *pw;                  // D
  u64 *x[2], *y[2];         // ping-pong GF vectors, 6 x (D + 1) and 6 x ((D + 1) / 2 + 1)
  u64 *small;               // 64 words: z, h0, h2, S, coef, r, zeta', tmp6, alpha, delta
  u64 *lhs, *rhs;           // 6 x (Dfinal + 1)
};

GfPlan plan_gf(Arena& a, long long nw, int R) {
  GfPlan g;
  g.D = 64 * nw;
  g.R = R < 0 ? default_R(g.D) : R;
  g.XA = a.take<u64>(6 * nw); g.YA = a.take<u64>(6 * nw); g.ZA = a.take<u64>(6 * nw);
  g.pw = a.take<u64>(g.D);
  g.x[0] = a.take<u64>(6 * (g.D + 1)); g.y[0] = a.take<u64>(6 * (g.D + 1));
  g.x[1] = a.take<u64>(6 * ((g.D + 1) / 2 + 1)); g.y[1] = a.take<u64>(6 * ((g.D + 1) / 2 + 1));
  g.small = a.take<u64>(128);
  const long long Df = dim_after(g.D, g.R);
  g.lhs = a.take<u64>(6 * (Df + 1)); g.rhs = a.take<u64>(6 * (Df + 1));
  return g;
}

// random shared GF element revealed with Pi_Rec (3 one-word messages, 3 hashes)
void gf_reveal(mpc_ctx* ctx, u32 purpose, u64 obj, u64* tmp6, u64* out) {
  launch_gf_random_shared(ctx->st, ctx->k01, ctx->k02, ctx->k12, purpose, obj, tmp6);
  launch_gf_rec1(ctx->st, tmp6, 0ull, out, ctx->status, ST_ABORT);
  g_launches += 2;
  count_msgs(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, 3, 8);
  count_msgs(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, 3, 32);
}

// secure GF inner product of (u, v) from their party sums (S must be zeroed by the caller, then
// filled by launch_gf_party_sums): finish + 3 one-word messages
void gf_inner_finish(mpc_ctx* ctx, const u64* S, u32 purpose, u64 obj, u64* h6) {
  launch_gf_inner_finish(ctx->st, S, ctx->k01, ctx->k02, purpose, obj, h6);
  g_launches += 1;
  count_msgs(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, 3, 8);
}

// Pi_MultVerify (Fig. PPEV) over GF(2^64) of the AND triples in g.XA/YA/ZA (batch 2)
int gf_verify(mpc_ctx* ctx, u64 vid, GfPlan& g, u64* trace) {
  cudaStream_t st = ctx->st;
  u64* z = g.small;          // 6
  u64* h0 = g.small + 8;     // 6
  u64* h2 = g.small + 16;    // 6
  u64* S = g.small + 24;     // 3
  u64* coef = g.small + 32;  // 5
  u64* r = g.small + 40;     // 1
  u64* zp = g.small + 41;    // 1
  u64* tmp6 = g.small + 48;  // 6
  u64* alpha = g.small + 56; // 6
  u64* dl = g.small + 64;    // 1
  u64* zn = g.small + 72;    // 6
  const long long nw = g.D / 64;
  CK(cudaMemsetAsync(g.small, 0, 128 * 8, st));
  gf_reveal(ctx, P_VER_R, make_obj(vid, 2, 0), tmp6, r);
  launch_gf_powers(st, r, g.D, g.pw);
  launch_gf_tran(st, g.XA, g.YA, g.ZA, nw, g.pw, g.D + 1, g.x[0], g.y[0], z);
  g_launches += 2;
  long long D = g.D;
  int cur = 0;
  const u64 X1 = 3ull, XX = 2ull;   // 1 + x and x: the fold weights at the third point x
  for (int k = 1; k <= g.R; ++k) {
    const long long cap = cur == 0 ? g.D + 1 : (g.D + 1) / 2 + 1;
    u64* xv = g.x[cur];
    u64* yv = g.y[cur];
    if (D & 1)
      for (int c = 0; c < 6; ++c) {
        CK(cudaMemsetAsync(xv + c * cap + D, 0, 8, st));
        CK(cudaMemsetAsync(yv + c * cap + D, 0, 8, st));
      }
    const long long Dh = (D + 1) / 2;
    const u64 obj = make_obj(vid, 2, (u32)k);
    const u64* uc[6];
    const u64* vc[6];
    for (int c = 0; c < 6; ++c) {
      uc[c] = xv + c * cap;
      vc[c] = yv + c * cap;
    }
    CK(cudaMemsetAsync(S, 0, 3 * 8, st));
    launch_gf_party_sums(st, uc, vc, Dh, 2, 0, 0, 0, 0, S);           // even entries
    g_launches += 1;
    gf_inner_finish(ctx, S, P_VER_H0, obj, h0);
    CK(cudaMemsetAsync(S, 0, 3 * 8, st));
    launch_gf_party_sums(st, uc, vc, Dh, 1, 0, 1, X1, XX, S);         // f(x) = (1+x) f(0) + x f(1)
    g_launches += 1;
    gf_inner_finish(ctx, S, P_VER_H2, obj, h2);
    gf_reveal(ctx, P_VER_ZETA, obj, tmp6, zp);
    launch_gf_lagrange(st, zp, coef);
    launch_gf_combine_z(st, coef, h0, h2, z, zn);
    g_launches += 2;
    CK(cudaMemcpyAsync(z, zn, 6 * 8, cudaMemcpyDeviceToDevice, st));
    const long long ocap = (g.D + 1) / 2 + 1;
    u64* xo = g.x[1];
    u64* yo = g.y[1];
    if (cur == 1) {   // fold in place is not allowed: fold into slot 0's storage
      xo = g.x[0];
      yo = g.y[0];
    }
    const long long ocap2 = cur == 1 ? g.D + 1 : ocap;
    launch_gf_fold6x2(st, xv, yv, cap, D, coef, xo, yo, ocap2);
    g_launches += 1;
    if (trace) {
      u64* t = trace + (long long)(k - 1) * MPC_TRACE_GF_ROUND;
      CK(cudaMemcpyAsync(t, zp, 8, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(t + 1, h0, 48, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(t + 7, h2, 48, cudaMemcpyDeviceToDevice, st));
    }
    cur ^= 1;
    D = Dh;
  }
  // Pi_InnerVerify (Fig. DPV): alpha random (kept shared), x' = x alpha, Delta = <[x'; alpha],
  // [y; -z]> opened, accept iff 0
  const long long cap = cur == 0 ? g.D + 1 : (g.D + 1) / 2 + 1;
  u64* xv = g.x[cur];
  u64* yv = g.y[cur];
  const u64 obj = make_obj(vid, 2, 0);
  launch_gf_random_shared(st, ctx->k01, ctx->k02, ctx->k12, P_VER_ALPHA, obj, alpha);
  g_launches += 1;
  const u64* xc[6];
  for (int c = 0; c < 6; ++c) xc[c] = xv + c * cap;
  const long long Df = D;
  launch_gf_mult_alpha(st, xc, alpha, Df, Df + 1, ctx->k01, ctx->k02, obj, g.lhs);
  g_launches += 1;
  count_msgs(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, 3, (u64)8 * Df);
  // lhs = [x alpha ; alpha], rhs = [y ; -z] (-z = z in characteristic 2), Df + 1 entries each
  for (int c = 0; c < 6; ++c) {
    CK(cudaMemcpyAsync(g.lhs + c * (Df + 1) + Df, alpha + c, 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(g.rhs + c * (Df + 1), yv + c * cap, (size_t)Df * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(g.rhs + c * (Df + 1) + Df, z + c, 8, cudaMemcpyDeviceToDevice, st));
  }
  const u64* uc[6];
  const u64* vc[6];
  for (int c = 0; c < 6; ++c) {
    uc[c] = g.lhs + c * (Df + 1);
    vc[c] = g.rhs + c * (Df + 1);
  }
  CK(cudaMemsetAsync(S, 0, 3 * 8, st));
  launch_gf_party_sums(st, uc, vc, Df + 1, 1, 0, 0, 0, 0, S);
  g_launches += 1;
  gf_inner_finish(ctx, S, P_VER_DELTA, obj, tmp6);
  launch_gf_rec1(st, tmp6, 0ull, dl, ctx->status, ST_ABORT);
  launch_gf_check_zero(st, dl, ctx->status, ST_VERIFY);
  g_launches += 2;
  count_msgs(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, 3, 8);
  count_msgs(ctx, MPC_PHASE_VERIFY, MPC_PROTO_VERIFY, 3, 32);
  if (trace) CK(cudaMemcpyAsync(trace + (long long)g.R * MPC_TRACE_GF_ROUND, dl, 8, cudaMemcpyDeviceToDevice, st));
  return cuda_check(ctx, "gf_verify");
}

struct NLPlan {
  int nst;
  CSPlan cs[2];
  u64 *a[2], *b[2], *o[2];       // stage operands (6 x np each)
  // batch 0: arithmetic products
  long long nm;
  u64 *MX, *MY, *MZ;
  VMultPlan vm;
  // batch 1: edaBit inner products (D1 = 64 sum np rows)
  long long ne, D1;
  int R1;
  Small s1;
  u64* pw1;
  Dense d1;
  IVBuf iv1;
  u64* Ye;                       // 6 x D1 ring words: the y side before its first fold
  u64* S6;                       // 6 x ne: the first round's per-element party-sum words
  u64* A1;                       // ne x 64: r^g f, the first round's x fold
  u64** ydev;                    // 6 device pointers (kernel argument)
  // batch 2: AND gates
  GfPlan gf;
  // batch 3: edaBit bit products (nb = 64 sum np), x only [r]_1 and y only [r]_2 (reading N9)
  long long nb;
  int Rb;
  Small sb;
  PowPlan ppb;
  u64* pwb;
  Dense db;
  IVBuf ivb;
  u64* Yb;                       // 2 x nb ring words: components 1 and 5 of the b2 bits
};

NLPlan plan_nl(Arena& a, int nst, const long long np[2]) {
  NLPlan p;
  p.nst = nst;
  p.nm = 0;
  p.ne = 0;
  long long andw = 0;
  for (int s = 0; s < nst; ++s) {
    p.a[s] = a.take<u64>(6 * np[s]);
    p.b[s] = a.take<u64>(6 * np[s]);
    p.o[s] = a.take<u64>(6 * np[s]);
    p.cs[s] = plan_cs(a, np[s]);
    p.nm += 3 * np[s];
    p.ne += np[s];
    andw += p.cs[s].and_words;
  }
  p.MX = a.take<u64>(6 * p.nm); p.MY = a.take<u64>(6 * p.nm); p.MZ = a.take<u64>(6 * p.nm);
  p.vm = plan_vmult(a, p.nm, -1);
  p.D1 = 64 * p.ne;
  p.R1 = default_R(p.D1);
  p.s1 = plan_small(a);
  p.pw1 = a.take<u64>(p.ne * 64);
  const bool xc[6] = {false, false, true, false, true, false};
  const bool yc[6] = {true, true, true, true, true, true};
  p.d1 = plan_dense(a, p.D1, xc, yc, p.R1, true);
  p.iv1 = plan_iv(a, dim_after(p.D1, p.R1));
  p.Ye = a.take<u64>(6 * p.D1);
  p.S6 = a.take<u64>(6 * p.ne);
  p.A1 = a.take<u64>(p.ne * 64);
  p.ydev = a.take<u64*>(6);
  p.gf = plan_gf(a, andw, -1);
  p.nb = 64 * p.ne;
  p.Rb = default_R(p.nb);
  p.sb = plan_small(a);
  p.pwb = a.take<u64>(p.nb * 64);
  p.ppb = plan_pow(a, p.nb);
  const bool bx[6] = {true, false, false, true, false, false};
  const bool by[6] = {false, true, false, false, false, true};
  p.db = plan_dense(a, p.nb, bx, by, p.Rb);
  p.ivb = plan_iv(a, dim_after(p.nb, p.Rb));
  p.Yb = a.take<u64>(2 * p.nb);
  return p;
}

// copy component c of an n-element sharing into a concatenated sharing of total length tot at
// offset off
int append_sharing(mpc_ctx* ctx, const u64* src, long long n, u64* dst, long long tot, long long off) {
  for (int c = 0; c < 6; ++c)
    CK(cudaMemcpyAsync(dst + c * tot + off, src + c * n, (size_t)n * 8, cudaMemcpyDeviceToDevice, ctx->st));
  return MPC_OK;
}

int verify_nl(mpc_ctx* ctx, u64 vid, NLPlan& p, u64* trace) {
  int rc;
  cudaStream_t st = ctx->st;
  // ---- batch 0: the daBit products (two) and the final product, stage by stage (the edaBit
  // bit products are batch 3)
  long long off = 0;
  for (int s = 0; s < p.nst; ++s) {
    CSPlan& c = p.cs[s];
    const u64* trip[3][3] = {{c.A1, c.A2, c.t}, {c.rpd, c.A3, c.u}, {c.d, c.gea, c.prod}};
    const long long len[3] = {c.np, c.np, c.np};
    for (int q = 0; q < 3; ++q) {
      if ((rc = append_sharing(ctx, trip[q][0], len[q], p.MX, p.nm, off))) return rc;
      if ((rc = append_sharing(ctx, trip[q][1], len[q], p.MY, p.nm, off))) return rc;
      if ((rc = append_sharing(ctx, trip[q][2], len[q], p.MZ, p.nm, off))) return rc;
      off += len[q];
    }
  }
  {
    VMultPlan& v = p.vm;
    const Small& s = v.s;
    const long long n = p.nm;
    reveal(ctx, P_VER_R, make_obj(vid, 0, 0), s.tmp6, s.r);
    if ((rc = power_table(ctx, s.r, v.pp, v.pw, s.aux))) return rc;
    Vec& x = v.dv.x[0];
    Vec ylift;
    for (int c = 0; c < 6; ++c) {
      launch_gr_scale_rows(st, v.pw, p.MX + c * n, n, x.c[c]);
      ylift.c[c] = p.MY + c * n;
    }
    CK(cudaMemsetAsync(s.zinit, 0, 384 * 8, st));
    launch_scalar_gr_sum(st, n, p.MZ, n, 6, v.pw, s.zinit);
    v.dv.cur = 0;
    if ((rc = run_dense(ctx, vid, 0, v.dv, n, s.zinit, 1, v.R, s, v.iv, trace, &ylift))) return rc;
  }
  u64* tr1 = trace ? trace + (long long)(p.vm.R + 1) * TRACE_ROUND : nullptr;
  // ---- batch 1: the edaBit inner products, weight r^e on row e (e over all stages)
  {
    const Small& s = p.s1;
    reveal(ctx, P_VER_R, make_obj(vid, 1, 0), s.tmp6, s.r);
    launch_gr_powers(st, s.r, p.ne, p.pw1);
    Vec ylift;
    for (int c = 0; c < 6; ++c) ylift.c[c] = p.Ye + c * p.D1;
    CK(cudaMemcpyAsync(p.ydev, ylift.c, 6 * sizeof(u64*), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(s.zinit, 0, 384 * 8, st));
    long long e0 = 0;
    for (int q = 0; q < p.nst; ++q) {   // the y words and the claim (x is never materialised)
      CSPlan& c = p.cs[q];
      launch_eda_tran(st, c.mbw, c.rp, c.np, p.pw1, e0, nullptr, nullptr, p.ydev);
      launch_scalar_gr_sum(st, c.np, c.ez, c.np, 6, p.pw1 + e0 * 64, s.zinit);
      g_launches += 1;
      e0 += c.np;
    }
    // Round 1 from the bits: x = r^g <m_i> pairs the bits 2k, 2k + 1 of one element, so the
    // party sums are sum_g r^g s(g) over per-element words (rows P1, P2 of each block; P0's are
    // zero) and the folded x is a selection among 0, r^g - r^g f, r^g f and r^g.
    CK(cudaMemsetAsync(s.S, 0, 4 * 192 * 8, st));
    e0 = 0;
    for (int q = 0; q < p.nst; ++q) {
      CSPlan& c = p.cs[q];
      launch_eda_r1_sums(st, c.mbw, c.rp, c.np, e0, p.ne, p.S6);
      g_launches += 1;
      e0 += c.np;
    }
    launch_scalar_gr_sum(st, p.ne, p.S6, p.ne, 2, p.pw1, s.S + 64);                   // S00
    launch_scalar_gr_sum(st, p.ne, p.S6 + 2 * p.ne, p.ne, 2, p.pw1, s.S + 192 + 64);  // S01 + S10
    launch_scalar_gr_sum(st, p.ne, p.S6 + 4 * p.ne, p.ne, 2, p.pw1, s.S + 576 + 64);  // S11
    round_tail(ctx, vid, 1, 1, s.zinit, s.z[1], s);
    Vec& xo = p.d1.x[1];
    Vec& yo = p.d1.y[1];
    if ((rc = gr_matmul(ctx, p.ne, p.pw1, nullptr, 1, 64, s.MM, nullptr, 0, p.A1, 64))) return rc;
    e0 = 0;
    for (int q = 0; q < p.nst; ++q) {
      CSPlan& c = p.cs[q];
      launch_eda_x_fold(st, c.mbw, c.np, e0, p.pw1, p.A1, xo.c[2], xo.c[4]);
      g_launches += 1;
      e0 += c.np;
    }
    const long long Dh = p.D1 / 2;
    for (int c = 0; c < 6; ++c) launch_fold_lifted(st, ylift.c[c], Dh, p.D1, s.coef, yo.c[c]);
    trace_round(ctx, tr1, 1, s);
    if ((rc = cuda_check(ctx, "edaBit first round"))) return rc;
    p.d1.cur = 1;
    if ((rc = run_dense(ctx, vid, 1, p.d1, Dh, s.z[1], 2, p.R1, s, p.iv1, tr1))) return rc;
  }
  u64* tr2 = tr1 ? tr1 + (long long)(p.R1 + 1) * TRACE_ROUND : nullptr;
  // ---- batch 2: every AND gate over GF(2^64), stage by stage, level by level
  {
    GfPlan& g = p.gf;
    const long long nw = g.D / 64;
    long long woff = 0;
    for (int s = 0; s < p.nst; ++s) {
      CSPlan& c = p.cs[s];
      for (int l = 1; l <= NL_LEVELS; ++l) {
        const long long lw = (long long)level_planes(l) * c.W;
        if ((rc = append_sharing(ctx, c.X[l], lw, g.XA, nw, woff))) return rc;
        if ((rc = append_sharing(ctx, c.Y[l], lw, g.YA, nw, woff))) return rc;
        if ((rc = append_sharing(ctx, c.Z[l], lw, g.ZA, nw, woff))) return rc;
        woff += lw;
      }
    }
    if ((rc = gf_verify(ctx, vid, g, tr2))) return rc;
  }
  u64* tr3 = tr2 ? tr2 + (long long)(p.gf.R + 1) * MPC_TRACE_GF_ROUND : nullptr;
  // ---- batch 3: the edaBit bit products b_{i,1} b_{i,2}, stage by stage (plane-major); x has
  // only the [r]_1 components and y only the [r]_2 ones, so the dense rounds take the
  // single-Gram form
  {
    const Small& s = p.sb;
    reveal(ctx, P_VER_R, make_obj(vid, 3, 0), s.tmp6, s.r);
    if ((rc = power_table(ctx, s.r, p.ppb, p.pwb, s.aux))) return rc;
    Vec& x = p.db.x[0];
    Vec ylift{};   // components 1 and 5 of the b2 bits, as ring words
    ylift.c[1] = p.Yb;
    ylift.c[5] = p.Yb + p.nb;
    CK(cudaMemsetAsync(s.zinit, 0, 384 * 8, st));
    long long e0 = 0;
    for (int q = 0; q < p.nst; ++q) {
      CSPlan& c = p.cs[q];
      const long long N = 64 * c.np;
      for (int comp : {0, 3})
        launch_gr_scale_rows(st, p.pwb + e0 * 64, c.B1 + comp * N, N, x.c[comp] + e0 * 64);
      for (int comp : {1, 5})
        CK(cudaMemcpyAsync(ylift.c[comp] + e0, c.B2 + comp * N, (size_t)N * 8,
                           cudaMemcpyDeviceToDevice, st));
      launch_scalar_gr_sum(st, N, c.eprod, N, 6, p.pwb + e0 * 64, s.zinit);
      e0 += N;
    }
    p.db.cur = 0;
    if ((rc = run_dense(ctx, vid, 3, p.db, p.nb, s.zinit, 1, p.Rb, s, p.ivb, tr3, &ylift)))
      return rc;
  }
  return MPC_OK;
}

int nl_finish(mpc_ctx* ctx) {
  u32 stv = 0;
  int rc = read_status(ctx, &stv);
  if (rc) return rc;
  if (stv & ST_ABORT) {
    ctx->aborted = true;
    return fail(ctx, MPC_ERR_ABORT, "Pi_Rec: inconsistent messages");
  }
  if (stv & ST_VERIFY) {
    ctx->aborted = true;
    return fail(ctx, MPC_ERR_VERIFY, "non-linear layer: verification failed");
  }
  return MPC_OK;
}

long long npad64(long long n) { return 64 * ((n + 63) / 64); }

void nl_plan_take(Arena& a, int nst, const long long np[2]) { plan_nl(a, nst, np); }

}  // namespace

int mpc_relu(mpc_ctx* ctx, uint64_t call_id, uint64_t verify_id, const uint64_t* xs, int64_t n,
             uint64_t* out, void* workspace, size_t workspace_bytes, uint64_t* trace) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (n <= 0) return fail(ctx, MPC_ERR_SHAPE, "relu: n <= 0");
  if (!xs || !out || !id_ok(call_id) || !id_ok(verify_id)) return fail(ctx, MPC_ERR_ARG, "relu: bad argument");
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  const long long np[2] = {npad64(n), 0};
  NLPlan p = plan_nl(ar, 1, np);
  if (!workspace || !ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "relu: workspace too small");
  Phase phase(ctx, MPC_PROF_NONLINEAR);
  cudaStream_t st = ctx->st;
  CK(cudaMemsetAsync(p.a[0], 0, (size_t)6 * np[0] * 8, st));
  CK(cudaMemsetAsync(p.b[0], 0, (size_t)6 * np[0] * 8, st));
  if ((rc = append_sharing(ctx, xs, n, p.a[0], np[0], 0))) return rc;      // zero-padded x, b = 0
  if ((rc = compare_select(ctx, call_id, 0, p.a[0], p.b[0], p.cs[0], p.o[0]))) return rc;
  if ((rc = verify_nl(ctx, verify_id, p, trace))) return rc;
  for (int c = 0; c < 6; ++c)
    CK(cudaMemcpyAsync(out + c * n, p.o[0] + c * np[0], (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
  if ((rc = cuda_check(ctx, "relu"))) return rc;
  return nl_finish(ctx);
}

int mpc_maxpool2(mpc_ctx* ctx, uint64_t call_id, uint64_t verify_id, const uint64_t* xs, int64_t B,
                 int64_t C, int64_t H, int64_t W, uint64_t* out, void* workspace,
                 size_t workspace_bytes, uint64_t* trace) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (B <= 0 || C <= 0 || H <= 0 || W <= 0 || (H & 1) || (W & 1))
    return fail(ctx, MPC_ERR_SHAPE, "maxpool2: bad shape");
  if (!xs || !out || !id_ok(call_id) || !id_ok(verify_id)) return fail(ctx, MPC_ERR_ARG, "maxpool2: bad argument");
  const long long nw = B * C * (H / 2) * (W / 2);
  Arena ar{(char*)workspace, workspace_bytes, 0, false};
  const long long np[2] = {npad64(2 * nw), npad64(nw)};
  NLPlan p = plan_nl(ar, 2, np);
  if (!workspace || !ar.ok()) return fail(ctx, MPC_ERR_WORKSPACE, "maxpool2: workspace too small");
  Phase phase(ctx, MPC_PROF_NONLINEAR);
  cudaStream_t st = ctx->st;
  for (int s = 0; s < 2; ++s) {
    CK(cudaMemsetAsync(p.a[s], 0, (size_t)6 * np[s] * 8, st));
    CK(cudaMemsetAsync(p.b[s], 0, (size_t)6 * np[s] * 8, st));
  }
  // stage 0 operands: left = [a ; c], right = [b ; d] of every window
  launch_window_gather(st, xs, B * C, H, W, np[0], p.a[0], p.b[0]);
  g_launches += 1;
  if ((rc = compare_select(ctx, call_id, 0, p.a[0], p.b[0], p.cs[0], p.o[0]))) return rc;
  for (int c = 0; c < 6; ++c) {
    CK(cudaMemcpyAsync(p.a[1] + c * np[1], p.o[0] + c * np[0], (size_t)nw * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(p.b[1] + c * np[1], p.o[0] + c * np[0] + nw, (size_t)nw * 8, cudaMemcpyDeviceToDevice, st));
  }
  if ((rc = compare_select(ctx, call_id, 1, p.a[1], p.b[1], p.cs[1], p.o[1]))) return rc;
  if ((rc = verify_nl(ctx, verify_id, p, trace))) return rc;
  for (int c = 0; c < 6; ++c)
    CK(cudaMemcpyAsync(out + c * nw, p.o[1] + c * np[1], (size_t)nw * 8, cudaMemcpyDeviceToDevice, st));
  if ((rc = cuda_check(ctx, "maxpool2"))) return rc;
  return nl_finish(ctx);
}

int mpc_hash_u64(mpc_ctx* ctx, const uint64_t* data, int64_t n, uint8_t* digest) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (n < 0) return fail(ctx, MPC_ERR_SHAPE, "hash: bad size");
  if ((n > 0 && !data) || !digest) return fail(ctx, MPC_ERR_ARG, "hash: bad argument");
  u32* scratch = nullptr;
  const size_t words = hash_scratch_words(n) + 8;
  cudaError_t e = cudaMalloc(&scratch, words * sizeof(u32));
  if (e != cudaSuccess) return fail(ctx, MPC_ERR_CUDA, "hash: scratch allocation");
  u32 h[8];
  launch_hash_u64(ctx->st, data, n, scratch, scratch + words - 8);
  e = cudaMemcpyAsync(h, scratch + words - 8, sizeof(h), cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  cudaFree(scratch);
  if (e != cudaSuccess) return fail(ctx, MPC_ERR_CUDA, cudaGetErrorString(e));
  for (int q = 0; q < 8; ++q)
    for (int b = 0; b < 4; ++b) digest[4 * q + b] = (uint8_t)(h[q] >> (24 - 8 * b));
  return cuda_check(ctx, "hash");
}

int mpc_gather(mpc_ctx* ctx, const uint64_t* xs, int64_t n_in, const int64_t* idx, int64_t n_out,
               uint64_t* out) {
  int rc = guard(ctx);
  if (rc) return rc;
  if (n_in <= 0 || n_out <= 0) return fail(ctx, MPC_ERR_SHAPE, "gather: bad size");
  if (!xs || !idx || !out) return fail(ctx, MPC_ERR_ARG, "gather: bad argument");
  launch_gather(ctx->st, xs, n_in, reinterpret_cast<const long long*>(idx), n_out, out);
  g_launches += 1;
  return cuda_check(ctx, "gather");
}
