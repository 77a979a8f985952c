// Elementwise and rearrangement kernels of the layer-level calls: the fixed-point encoding and
// decoding of Sec. 2 Notation (mpc_share_fixed, mpc_reconstruct_fixed), the im2col lowering of a
// convolution to one inner product per output (Sec. 4.1, mpc_conv2d), and the two local steps of
// a standalone truncation (Fig. trunc, mpc_trunc): the mask-switch messages and the online shift.
//
// Sharing layout: component c of an n-element sharing at [c n, (c + 1) n):
//   0: P0.[r]_1   1: P0.[r]_2   2: P1.m   3: P1.[r]_1   4: P2.m   5: P2.[r]_2
#include "kernels.h"

namespace mpc3 {

namespace {

constexpr int LTPB = 256;

inline unsigned lgrid(long long n) {
  long long g = (n + LTPB - 1) / LTPB;
  if (g > (1ll << 20)) g = 1ll << 20;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// floor(x 2^k) as a two's-complement word; x 2^k outside [-2^63, 2^63) saturates, NaN gives 0.
// Scaling by 2^k is exact in binary floating point (short of overflow, which saturates), and so
// is floor; the conversion is exact inside the range.
__global__ void k_encode_fixed(const double* __restrict__ x, long long n, int k,
                               u64* __restrict__ out) {
  const double lo = -9223372036854775808.0, hi = 9223372036854775808.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = floor(ldexp(x[i], k));
    long long w;
    if (v >= lo && v < hi) w = (long long)v;
    else if (v >= hi) w = 0x7FFFFFFFFFFFFFFFll;
    else if (v < lo) w = (long long)0x8000000000000000ull;
    else w = 0;   // NaN
    out[i] = (u64)w;
  }
}

// the signed value of a word divided by 2^k
__global__ void k_decode_fixed(const u64* __restrict__ v, long long n, int k,
                               double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = ldexp((double)(long long)v[i], -k);
}

// cols[c][row][col] = x[c][b][ch][i s + di - p][j s + dj - p] (0 outside the image) for every
// share component c, row = (b Ho + i) Wo + j, col = (ch kh + di) kw + dj.
__global__ void k_im2col(const u64* __restrict__ x, ConvGeom g, u64* __restrict__ cols) {
  const long long Mr = (long long)g.B * g.Ho * g.Wo, Kc = (long long)g.C * g.kh * g.kw;
  const long long n_in = (long long)g.B * g.C * g.H * g.W, per = Mr * Kc, total = 6 * per;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long comp = t / per, rc = t - comp * per;
    const long long row = rc / Kc, col = rc - row * Kc;
    const long long j = row % g.Wo, i = (row / g.Wo) % g.Ho, b = row / ((long long)g.Wo * g.Ho);
    const long long dj = col % g.kw, di = (col / g.kw) % g.kh, ch = col / ((long long)g.kw * g.kh);
    const long long y = i * g.stride + di - g.pad, z = j * g.stride + dj - g.pad;
    u64 v = 0;
    if (y >= 0 && y < g.H && z >= 0 && z < g.W)
      v = x[comp * n_in + ((b * g.C + ch) * g.H + y) * g.W + z];
    cols[t] = v;
  }
}

// d1 = [r_x]_1 - [r]_1 and d2 = [r_x]_2 - [r]_2, as P1 and P2 compute them (components 3, 5)
// and as P0 does (components 0, 1); rx holds the pairs' mask shares in the same components.
__global__ void k_trunc_remask(const u64* __restrict__ xs, const u64* __restrict__ rx, long long n,
                               u64* __restrict__ d1_p1, u64* __restrict__ d2_p2,
                               u64* __restrict__ d1_p0, u64* __restrict__ d2_p0) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    d1_p1[i] = rx[3 * n + i] - xs[3 * n + i];
    d2_p2[i] = rx[5 * n + i] - xs[5 * n + i];
    d1_p0[i] = rx[i] - xs[i];
    d2_p0[i] = rx[n + i] - xs[n + i];
  }
}

// m' = m + d1 + d2 = x + r_x at P1 (own d1, received d2) and P2 (received d1, own d2);
// m_z = m' >>_arith t into the m components of out (its masks are the pairs' r_z).
__global__ void k_trunc_online(const u64* __restrict__ xs, long long n, const u64* __restrict__ d1,
                               const u64* __restrict__ d2_at_p1, const u64* __restrict__ d1_at_p2,
                               const u64* __restrict__ d2, int t, u64* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const u64 m1 = xs[2 * n + i] + d1[i] + d2_at_p1[i];
    const u64 m2 = xs[4 * n + i] + d1_at_p2[i] + d2[i];
    out[2 * n + i] = (u64)(((long long)m1) >> t);
    out[4 * n + i] = (u64)(((long long)m2) >> t);
  }
}

}  // namespace

void launch_encode_fixed(cudaStream_t st, const double* x, long long n, int k, u64* out) {
  if (n <= 0) return;
  k_encode_fixed<<<lgrid(n), LTPB, 0, st>>>(x, n, k, out);
}

void launch_decode_fixed(cudaStream_t st, const u64* v, long long n, int k, double* out) {
  if (n <= 0) return;
  k_decode_fixed<<<lgrid(n), LTPB, 0, st>>>(v, n, k, out);
}

void launch_im2col(cudaStream_t st, const u64* x, const ConvGeom& g, u64* cols) {
  const long long total = 6ll * g.B * g.Ho * g.Wo * g.C * g.kh * g.kw;
  if (total <= 0) return;
  k_im2col<<<lgrid(total), LTPB, 0, st>>>(x, g, cols);
}

void launch_trunc_remask(cudaStream_t st, const u64* xs, const u64* rx, long long n, u64* d1_p1,
                         u64* d2_p2, u64* d1_p0, u64* d2_p0) {
  if (n <= 0) return;
  k_trunc_remask<<<lgrid(n), LTPB, 0, st>>>(xs, rx, n, d1_p1, d2_p2, d1_p0, d2_p0);
}

void launch_trunc_online(cudaStream_t st, const u64* xs, long long n, const u64* d1,
                         const u64* d2_at_p1, const u64* d1_at_p2, const u64* d2, int t,
                         u64* out) {
  if (n <= 0) return;
  k_trunc_online<<<lgrid(n), LTPB, 0, st>>>(xs, n, d1, d2_at_p1, d1_at_p2, d2, t, out);
}

}  // namespace mpc3

// ---- test hook: a bounded wait that runs out -------------------------------------------------
#include "tcgen05.cuh"

namespace mpc3 {
namespace {

// One thread waits, with the tensor-core kernels' bounded-wait helper and a limit of `cycles`,
// on an mbarrier that nothing arrives at; on expiry it records err_flag in the status word and
// returns, exactly as a tensor-core kernel's waiting role does.
__global__ void k_wait_expires(long long cycles, unsigned* __restrict__ err, unsigned err_flag) {
  __shared__ __align__(8) u64 bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 1);
  abort_flag = 0;
  tc::mbar_init_fence();
  if (!tc::mbar_wait(&bar, 0u, &abort_flag, cycles)) atomicOr(err, err_flag);
}

}  // namespace

void launch_wait_expires(cudaStream_t st, long long cycles, unsigned* err, unsigned err_flag) {
  k_wait_expires<<<1, 32, 0, st>>>(cycles, err, err_flag);
}

}  // namespace mpc3
