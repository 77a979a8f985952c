// Pi_Rec for callers that cannot allocate device memory when they reconstruct.
//
// mpc_reconstruct() takes its scratch (the three shares each party receives, and the hash
// scratch) from a workspace the caller allocates.  Some callers cannot do that at the moment they
// reconstruct: a serving loop that has handed all free device memory to its own pool, code that
// must not call the CUDA allocator because cudaMalloc/cudaFree may synchronise the whole device
// and stall the other streams, or code that links libmpc3 without any device allocator at all.
// mpc_reconstruct_noalloc() runs the same protocol (same messages, hashes, checks and opening)
// with that scratch in one fixed array compiled into this file instead.  It allocates nothing.
//
// The array is a file-scope __device__ variable, so every GPU that loads the library holds it
// (sizeof(NoallocScratch), about 6 MiB) until the process exits.  Host code cannot use its name
// as a device address; its address is resolved per device with cudaGetSymbolAddress() the first
// time the entry point runs on that device (with that device current), and passed to the kernels.
// Every call shares the array: calls that can overlap on the GPU (other streams, other contexts
// on the same device) race on it and must be serialised by the caller.  Every word a call reads
// is written earlier in the same call, so nothing needs clearing between calls.
#include <cstring>
#include <mutex>
#include <string>

#include "mpc3.h"
#include "kernels.h"

namespace mpc3 {
namespace internal {
int ctx_guard(mpc_ctx* c);
int ctx_fail(mpc_ctx* c, int code, const char* msg);
int ctx_deliver(mpc_ctx* c, int phase, int proto, const u64* src, u64* dst, long long n, int site);
void ctx_count(mpc_ctx* c, int phase, int proto, int count, u64 bytes_each);
int ctx_read_status(mpc_ctx* c, u32* out);
bool ctx_has_pending(const mpc_ctx* c);
cudaStream_t ctx_stream(const mpc_ctx* c);
u32* ctx_status_word(const mpc_ctx* c);
void ctx_set_aborted(mpc_ctx* c);
}  // namespace internal
}  // namespace mpc3

using namespace mpc3;
using namespace mpc3::internal;

namespace {

constexpr long long kMaxN = MPC_NOALLOC_MAX_N;
constexpr long long kHashWords = hash_scratch_words_for(kMaxN);   // 32-bit words per hash

struct NoallocScratch {
  u64 in_p2_r1[kMaxN];      // [r]_1 as received by P2 from P0
  u64 in_p1_r2[kMaxN];      // [r]_2 as received by P1 from P0
  u64 in_p0_m[kMaxN];       // m as received by P0 from P1
  u32 hs[6][kHashWords];    // Merkle scratch of the six hashes
  u32 dg[6 * 8];            // the six digests
};

static __device__ __align__(256) NoallocScratch g_noalloc;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoallocScratch* g_addr[kMaxDevices] = {};

// Device address of g_noalloc on the current device (resolved once per device).
int scratch_for_current_device(mpc_ctx* ctx, NoallocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ctx_fail(ctx, MPC_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return ctx_fail(ctx, MPC_ERR_ARG, "device ordinal too large");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc);
    if (e != cudaSuccess || !p)
      return ctx_fail(ctx, MPC_ERR_CUDA,
                      (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
    g_addr[dev] = static_cast<NoallocScratch*>(p);
  }
  *out = g_addr[dev];
  return MPC_OK;
}

}  // namespace

extern "C" int mpc_reconstruct_noalloc(mpc_ctx* ctx, const uint64_t* xs, int64_t n,
                                       uint64_t* out) {
  int rc = ctx_guard(ctx);   // also makes the context's device current
  if (rc) return rc;
  if (!xs || !out) return ctx_fail(ctx, MPC_ERR_ARG, "reconstruct_noalloc: null pointer");
  if (n <= 0 || n > kMaxN)
    return ctx_fail(ctx, MPC_ERR_SHAPE,
                    "reconstruct_noalloc: n must be in [1, MPC_NOALLOC_MAX_N = 262144]");
  if (ctx_has_pending(ctx))
    return ctx_fail(ctx, MPC_ERR_PENDING, "reconstruct_noalloc: products are not verified yet");
  NoallocScratch* s = nullptr;
  if ((rc = scratch_for_current_device(ctx, &s))) return rc;
  cudaStream_t st = ctx_stream(ctx);
  const int ph = MPC_PHASE_ONLINE, pr = MPC_PROTO_REC;
  if ((rc = ctx_deliver(ctx, ph, pr, xs, s->in_p2_r1, n, -1))) return rc;                // P0 -> P2
  if ((rc = ctx_deliver(ctx, ph, pr, xs + n, s->in_p1_r2, n, MPC_SITE_REC_MSG))) return rc;  // P0 -> P1
  if ((rc = ctx_deliver(ctx, ph, pr, xs + 2 * n, s->in_p0_m, n, -1))) return rc;         // P1 -> P0
  u32* d = s->dg;
  launch_hash_u64(st, xs + 3 * n, n, s->hs[0], d + 0);     // P1: H([r]_1) -> P2
  launch_hash_u64(st, xs + 4 * n, n, s->hs[1], d + 8);     // P2: H(m) -> P0
  launch_hash_u64(st, xs + 5 * n, n, s->hs[2], d + 16);    // P2: H([r]_2) -> P1
  ctx_count(ctx, ph, pr, 3, 32);
  launch_hash_u64(st, s->in_p2_r1, n, s->hs[3], d + 24);   // P2 hashes the [r]_1 it received
  launch_hash_u64(st, s->in_p0_m, n, s->hs[4], d + 32);    // P0 hashes the m it received
  launch_hash_u64(st, s->in_p1_r2, n, s->hs[5], d + 40);   // P1 hashes the [r]_2 it received
  launch_digest_check(st, d + 0, d + 24, d + 8, d + 32, d + 16, d + 40, ctx_status_word(ctx), 1u);
  launch_open_p1(st, xs + 2 * n, xs + 3 * n, s->in_p1_r2, n, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_fail(ctx, MPC_ERR_CUDA, cudaGetErrorString(e));
  u32 stv = 0;
  if ((rc = ctx_read_status(ctx, &stv))) return rc;
  if (stv & 1u) {
    ctx_set_aborted(ctx);
    cudaMemsetAsync(out, 0, (size_t)n * 8, st);
    return ctx_fail(ctx, MPC_ERR_ABORT, "Pi_Rec: inconsistent messages");
  }
  return MPC_OK;
}
