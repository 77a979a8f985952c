// Elementwise protocol kernels: input sharing (Pi_<.>^{l,0}), Pi_Mult offline/online (Fig. MultP),
// the m-share exchange finish with the online truncation m >> t (Fig. trunc, online), and the
// truncation-pair preprocessing (Fig. trunc, preprocessing).
//
// Sharing layout: a <.>-shared tensor of n elements is 6n words, component c at [c*n, (c+1)*n):
//   0: P0.[r]_1   1: P0.[r]_2   2: P1.m   3: P1.[r]_1   4: P2.m   5: P2.[r]_2
// Each thread owns 8 consecutive elements, i.e. one ChaCha20 block per PRG stream it draws.
#include "kernels.h"

namespace mpc3 {

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(long long n8) {
  long long g = (n8 + TPB - 1) / TPB;
  if (g > (1ll << 20)) g = 1ll << 20;
  if (g < 1) g = 1;
  return (unsigned)g;
}

__device__ __forceinline__ u64 asr64(u64 v, int t) { return (u64)(((long long)v) >> t); }

// Words 8 blk .. 8 blk + 7 of a truncation-bit stream.  Unkeyed: words of the stream (tag, obj).
// Keyed by rows (row_keys != null, outputs row-major with N per row): word e is word e mod N of
// the stream (tag, row_keys[e / N]), so that a row draws the same bits whatever batch it is in;
// words past E are 0.
__device__ __forceinline__ void bits_block8(const Key& key, u32 tag, u64 obj, u64 blk,
                                            const u64* __restrict__ row_keys, long long N,
                                            long long E, u64 w[8]) {
  if (!row_keys) {
    prf_block8(key, tag, obj, blk, w);
    return;
  }
#pragma unroll 1
  for (int j = 0; j < 8; ++j) {
    const long long e = (long long)blk * 8 + j;
    w[j] = 0;
    if (e < E) {
      const long long row = e / N, col = e - row * N;
      u64 b8[8];
      prf_block8(key, tag, row_keys[row], (u64)(col >> 3), b8);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q == (int)(col & 7)) w[j] = b8[q];
    }
  }
}

// v, with a compiler scheduling fence: code that uses the result is not hoisted above the memory
// operations before it (keeps one ChaCha20 block live at a time)
__device__ __forceinline__ u64 seq_u64(u64 v) {
  u64 r;
  asm volatile("mov.b64 %0, %1;\n" : "=l"(r) : "l"(v) : "memory");
  return r;
}

// Warp-cooperative transfers of 8 consecutive elements per lane (lane l owns elements
// e0 + 8 l .. e0 + 8 l + 7), staged through a per-warp shared block (32 x 9 words) so that every
// global access instruction covers 32 consecutive words.  All 32 lanes must call them together.
__device__ __forceinline__ void store8w(u64* __restrict__ out, long long e0, long long n,
                                        const u64 v[8], u64* st) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 8; ++j) st[lane * 9 + j] = v[j];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int idx = j * 32 + lane;
    if (e0 + idx < n) out[e0 + idx] = st[(idx >> 3) * 9 + (idx & 7)];
  }
  __syncwarp();
}
__device__ __forceinline__ void load8w(const u64* __restrict__ in, long long e0, long long n,
                                       u64 v[8], u64* st) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int idx = j * 32 + lane;
    st[(idx >> 3) * 9 + (idx & 7)] = (e0 + idx < n) ? in[e0 + idx] : 0ull;
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = st[lane * 9 + j];
  __syncwarp();
}

// Pi_<.>^{l,0}(x): [r]_1 from eta01 (P0, P1), [r]_2 from eta02 (P0, P2); P0 forms
// m = x + [r]_1 + [r]_2 (its outgoing message to P1 and P2).
__global__ void __launch_bounds__(TPB)
k_share_input(const u64* __restrict__ x, long long n, Key k01, Key k02, u32 tag1, u32 tag2,
              u64 obj, u64* __restrict__ s, u64* __restrict__ m_out) {
  __shared__ u64 stage[TPB / 32][32 * 9];
  u64* st = stage[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const long long nb = (n + 7) / 8;
  for (long long bw = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); bw < nb;
       bw += (long long)gridDim.x * blockDim.x) {
    const u64 b = (u64)(bw + lane);
    const long long e0 = bw * 8;
    u64 r1[8], r2[8], xv[8];
    prf_block8(k01, tag1, obj, b, r1);
    prf_block8(k02, tag2, obj, b, r2);
    store8w(s, e0, n, r1, st);
    store8w(s + n, e0, n, r2, st);
    store8w(s + 3 * n, e0, n, r1, st);
    store8w(s + 5 * n, e0, n, r2, st);
    load8w(x, e0, n, xv, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) xv[j] += r1[j] + r2[j];
    store8w(m_out, e0, n, xv, st);
  }
}

// [r] <- Pi_[.] (random) into the mask components of a sharing (output wires of Pi_Mult / Pi_Inner).
__global__ void __launch_bounds__(TPB)
k_fill_masks(long long n, Key k01, Key k02, u32 tag1, u32 tag2, u64 obj, u64* __restrict__ s) {
  __shared__ u64 stage[TPB / 32][32 * 9];
  u64* st = stage[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const long long nb = (n + 7) / 8;
  for (long long bw = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); bw < nb;
       bw += (long long)gridDim.x * blockDim.x) {
    const u64 b = (u64)(bw + lane);
    const long long e0 = bw * 8;
    u64 r1[8], r2[8];
    prf_block8(k01, tag1, obj, b, r1);
    prf_block8(k02, tag2, obj, b, r2);
    store8w(s, e0, n, r1, st);
    store8w(s + n, e0, n, r2, st);
    store8w(s + 3 * n, e0, n, r1, st);
    store8w(s + 5 * n, e0, n, r2, st);
  }
}

// Pi_Mult preprocessing (P0): [r_z] <- Pi_[.]; Gamma = r_x r_y + r_z; [Gamma]_1 = PRG(eta01);
// the message to P2 is [Gamma]_2 = Gamma - [Gamma]_1.
__global__ void k_mult_offline(const u64* __restrict__ xs, const u64* __restrict__ ys,
                               long long n, Key k01, Key k02, u32 tr1, u32 tr2, u32 tg1, u64 obj,
                               u64* __restrict__ zs, u64* __restrict__ g2_out) {
  const long long nb = (n + 7) / 8;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
       b += (long long)gridDim.x * blockDim.x) {
    u64 r1[8], r2[8], g1[8];
    prf_block8(k01, tr1, obj, (u64)b, r1);
    prf_block8(k02, tr2, obj, (u64)b, r2);
    prf_block8(k01, tg1, obj, (u64)b, g1);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long i = b * 8 + j;
      if (i < n) {
        const u64 rx = xs[i] + xs[n + i];
        const u64 ry = ys[i] + ys[n + i];
        const u64 gamma = rx * ry + r1[j] + r2[j];
        g2_out[i] = gamma - g1[j];
        zs[i] = r1[j];
        zs[n + i] = r2[j];
        zs[3 * n + i] = r1[j];
        zs[5 * n + i] = r2[j];
      }
    }
  }
}

// Pi_Mult online: P1: [m_z]_1 = -m_x [r_y]_1 - m_y [r_x]_1 + [Gamma]_1;
//                 P2: [m_z]_2 = m_x m_y - m_x [r_y]_2 - m_y [r_x]_2 + [Gamma]_2 (received).
__global__ void k_mult_online(const u64* __restrict__ xs, const u64* __restrict__ ys,
                              long long n, Key k01, u32 tg1, u64 obj,
                              const u64* __restrict__ g2_in, u64* __restrict__ p1_out,
                              u64* __restrict__ p2_out) {
  const long long nb = (n + 7) / 8;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
       b += (long long)gridDim.x * blockDim.x) {
    u64 g1[8];
    prf_block8(k01, tg1, obj, (u64)b, g1);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long i = b * 8 + j;
      if (i < n) {
        const u64 mx1 = xs[2 * n + i], rx1 = xs[3 * n + i];
        const u64 my1 = ys[2 * n + i], ry1 = ys[3 * n + i];
        p1_out[i] = g1[j] - mx1 * ry1 - my1 * rx1;
        const u64 mx2 = xs[4 * n + i], rx2 = xs[5 * n + i];
        const u64 my2 = ys[4 * n + i], ry2 = ys[5 * n + i];
        p2_out[i] = mx2 * my2 - mx2 * ry2 - my2 * rx2 + g2_in[i];
      }
    }
  }
}

// After the exchange: P1 holds m = own + received, P2 likewise.  With t >= 0 the truncated
// output's m is m >>_arith t (Fig. trunc, online), written into outs (P1.m, P2.m components).
__global__ void k_exchange_finish(long long n, const u64* __restrict__ p1_own,
                                  const u64* __restrict__ p1_in, const u64* __restrict__ p2_own,
                                  const u64* __restrict__ p2_in, u64* __restrict__ zs, int t,
                                  u64* __restrict__ outs) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const u64 m1 = p1_own[i] + p1_in[i];
    const u64 m2 = p2_in[i] + p2_own[i];
    zs[2 * n + i] = m1;
    zs[4 * n + i] = m2;
    if (outs) {
      outs[2 * n + i] = asr64(m1, t);
      outs[4 * n + i] = asr64(m2, t);
    }
  }
}

// Pi_Trunc^t preprocessing, P0's part plus every party's PRG draws.  Per output e:
//   b1 (eta01) and b2 (eta02) hold the bits b_{1,j}, b_{2,j};
//   Pi_Inner #1 (r_x): x_j = -2^(j+1) <b1_j>, y_j = <b2_j>, z = <p>, p = -2 (b1 & b2);
//   Pi_Inner #2 (r_z): x_j = c'_j <b1_j>, y_j = <b2_j>, z = <q>, q = -2 asr(b1 & b2, t);
// the bit sharings have m = 0, so P1's and P2's cross terms vanish and [m]_j = [Gamma]_j.
// P0's additive shares: [r_x]_1 = Gamma_p + b1 - [r_p]_1, [r_x]_2 = b2 - [r_p]_2 (and the same for
// r_z with asr(b1, t), asr(b2, t), Gamma_q, r_q).
// pq layout: <p> at pq[0..6E), <q> at pq[6E..12E).
__global__ void __launch_bounds__(TPB, 1)
k_trunc_p0(long long E, Key k01, Key k02, u64 obj, const u64* __restrict__ row_keys, long long N,
           int t, u32 ttb1, u32 ttb2,
           u32 tp1, u32 tp2, u32 tpg, u32 tq1, u32 tq2, u32 tqg,
           u64* __restrict__ zpre, u64* __restrict__ zout, u64* __restrict__ pq,
           u64* __restrict__ gp2_out, u64* __restrict__ gq2_out,
           u64* __restrict__ mp1_out, u64* __restrict__ mq1_out) {
  __shared__ u64 stage[TPB / 32][32 * 9];
  u64* st = stage[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const long long nb = (E + 7) / 8;
  u64* p = pq;
  u64* q = pq + 6 * E;
  // one stream at a time (few registers live); gamma_p = -2a + r_p1 + r_p2 with a = b1 & b2, so
  // [r_x]_1 = gamma_p + b1 - r_p1 = b1 - 2a + r_p2 (and the same for q with asr(., t))
  for (long long bw = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); bw < nb;
       bw += (long long)gridDim.x * blockDim.x) {
    const u64 b = (u64)(bw + lane);
    const long long e0 = bw * 8;
    u64 b1[8], b2[8], x[8], g[8];
    bits_block8(k01, ttb1, obj, b, row_keys, N, E, b1);
    bits_block8(k02, ttb2, obj, b, row_keys, N, E, b2);
    // <p>
    prf_block8(k01, tp1, obj, seq_u64(b), x);   // r_p1: P0 and P1 copies
    store8w(p, e0, E, x, st);
    store8w(p + 3 * E, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) g[j] = x[j] - 2 * (b1[j] & b2[j]);
    prf_block8(k02, tp2, obj, seq_u64(b), x);   // r_p2: P0 and P2 copies
    store8w(p + E, e0, E, x, st);
    store8w(p + 5 * E, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      g[j] += x[j];
      x[j] = b1[j] - 2 * (b1[j] & b2[j]) + x[j];   // [r_x]_1 = b1 - 2a + r_p2
    }
    store8w(zpre, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = b2[j] - (x[j] - b1[j] + 2 * (b1[j] & b2[j]));   // [r_x]_2 = b2 - r_p2
    store8w(zpre + E, e0, E, x, st);
    prf_block8(k01, tpg, obj, seq_u64(b), x);   // P1's [m_p]_1 = [Gamma_p]_1 (its own PRG draw)
    store8w(mp1_out, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = g[j] - x[j];
    store8w(gp2_out, e0, E, x, st);
    // <q>
    prf_block8(k01, tq1, obj, seq_u64(b), x);
    store8w(q, e0, E, x, st);
    store8w(q + 3 * E, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) g[j] = x[j] - 2 * asr64(b1[j] & b2[j], t);
    prf_block8(k02, tq2, obj, seq_u64(b), x);
    store8w(q + E, e0, E, x, st);
    store8w(q + 5 * E, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      g[j] += x[j];
      x[j] = asr64(b1[j], t) - 2 * asr64(b1[j] & b2[j], t) + x[j];   // [r_z]_1
    }
    store8w(zout, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j)   // [r_z]_2 = asr(b2, t) - r_q2
      x[j] = asr64(b2[j], t) - (x[j] - asr64(b1[j], t) + 2 * asr64(b1[j] & b2[j], t));
    store8w(zout + E, e0, E, x, st);
    prf_block8(k01, tqg, obj, seq_u64(b), x);
    store8w(mq1_out, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = g[j] - x[j];
    store8w(gq2_out, e0, E, x, st);
  }
}

// Pi_Trunc^t preprocessing, P1's and P2's part after the messages: m_p = [m_p]_1 + [m_p]_2 at each
// of P1, P2; [r_x]_1 := m_{r_x} - [r_{r_x}]_1 at P1, [r_x]_2 := -[r_{r_x}]_2 at P2 (same for r_z).
__global__ void __launch_bounds__(TPB, 2)
k_trunc_finish(long long E, Key k01, Key k02, u64 obj, const u64* __restrict__ row_keys,
               long long N, int t, u32 ttb1,
               u32 ttb2, const u64* __restrict__ p1_in_mp,
               const u64* __restrict__ p1_in_mq, const u64* __restrict__ p2_in_mp,
               const u64* __restrict__ p2_in_mq, const u64* __restrict__ p2_gp2,
               const u64* __restrict__ p2_gq2, const u64* __restrict__ p1_mp1,
               const u64* __restrict__ p1_mq1, u64* __restrict__ zpre,
               u64* __restrict__ zout, u64* __restrict__ pq) {
  __shared__ u64 stage[TPB / 32][32 * 9];
  u64* st = stage[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const long long nb = (E + 7) / 8;
  u64* p = pq;
  u64* q = pq + 6 * E;
  for (long long bw = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); bw < nb;
       bw += (long long)gridDim.x * blockDim.x) {
    const u64 b = (u64)(bw + lane);
    const long long e0 = bw * 8;
    u64 bb[8], m[8], x[8];
    bits_block8(k01, ttb1, obj, b, row_keys, N, E, bb);   // b1 (P1)
    // P1: m_p, m_q and its [r_x]_1, [r_z]_1
    load8w(p1_mp1, e0, E, m, st);
    load8w(p1_in_mp, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) m[j] += x[j];
    store8w(p + 2 * E, e0, E, m, st);
    load8w(p + 3 * E, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) m[j] = m[j] + bb[j] - x[j];
    store8w(zpre + 3 * E, e0, E, m, st);
    load8w(p1_mq1, e0, E, m, st);
    load8w(p1_in_mq, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) m[j] += x[j];
    store8w(q + 2 * E, e0, E, m, st);
    load8w(q + 3 * E, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) m[j] = m[j] + asr64(bb[j], t) - x[j];
    store8w(zout + 3 * E, e0, E, m, st);
    // P2
    bits_block8(k02, ttb2, obj, b, row_keys, N, E, bb);   // b2 (P2)
    load8w(p2_in_mp, e0, E, m, st);
    load8w(p2_gp2, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) m[j] += x[j];
    store8w(p + 4 * E, e0, E, m, st);
    load8w(p + 5 * E, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) m[j] = bb[j] - x[j];
    store8w(zpre + 5 * E, e0, E, m, st);
    load8w(p2_in_mq, e0, E, m, st);
    load8w(p2_gq2, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) m[j] += x[j];
    store8w(q + 4 * E, e0, E, m, st);
    load8w(q + 5 * E, e0, E, x, st);
#pragma unroll
    for (int j = 0; j < 8; ++j) m[j] = asr64(bb[j], t) - x[j];
    store8w(zout + 5 * E, e0, E, m, st);
  }
}

__global__ void k_xor_one(u64* p, u64 mask) { *p ^= mask; }

// words off .. off + n - 1 of a row-keyed truncation-bit stream (see bits_block8) into out
__global__ void k_prf_words_keyed(long long n, long long off, Key key, u32 tag,
                                  const u64* __restrict__ row_keys, long long N,
                                  u64* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = off + i, row = e / N, col = e - row * N;
    u64 b8[8];
    prf_block8(key, tag, row_keys[row], (u64)(col >> 3), b8);
    u64 w = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q == (int)(col & 7)) w = b8[q];
    out[i] = w;
  }
}

// stream words off .. off + n - 1 (block b holds words 8b .. 8b + 7) into out[0 .. n)
__global__ void k_prf_words(long long n, long long off, Key key, u32 tag, u64 obj,
                            u64* __restrict__ out) {
  const long long b0 = off / 8, nb = (off + n + 7) / 8 - b0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = b0 + i;
    u64 w[8];
    prf_block8(key, tag, obj, (u64)b, w);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long g = b * 8 + j - off;
      if (g >= 0 && g < n) out[g] = w[j];
    }
  }
}

// x = m - [r]_1 - [r]_2 from P1's view (own m, own [r]_1, received [r]_2).
__global__ void k_open_p1(const u64* __restrict__ m, const u64* __restrict__ r1,
                          const u64* __restrict__ r2, long long n, u64* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = m[i] - r1[i] - r2[i];
}

}  // namespace

void launch_share_input(cudaStream_t st, const u64* x, long long n, Key k01, Key k02, u64 obj,
                        u64* s6, u64* p0_out_m) {
  if (n <= 0) return;
  k_share_input<<<grid_for((n + 7) / 8), TPB, 0, st>>>(x, n, k01, k02, make_tag(P_SHARE, C_R1),
                                                       make_tag(P_SHARE, C_R2), obj, s6, p0_out_m);
}

void launch_fill_masks(cudaStream_t st, long long n, Key k01, Key k02, u32 purpose, u64 obj,
                       u64* s6) {
  if (n <= 0) return;
  k_fill_masks<<<grid_for((n + 7) / 8), TPB, 0, st>>>(n, k01, k02, make_tag(purpose, C_R1),
                                                      make_tag(purpose, C_R2), obj, s6);
}

void launch_mult_offline(cudaStream_t st, const u64* xs, const u64* ys, long long n, Key k01,
                         Key k02, u64 obj, u64* zs, u64* p0_out_g2) {
  if (n <= 0) return;
  k_mult_offline<<<grid_for((n + 7) / 8), TPB, 0, st>>>(
      xs, ys, n, k01, k02, make_tag(P_MULT, C_R1), make_tag(P_MULT, C_R2),
      make_tag(P_MULT, C_G1), obj, zs, p0_out_g2);
}

void launch_mult_offline_p(cudaStream_t st, const u64* xs, const u64* ys, long long n, Key k01,
                           Key k02, u32 purpose, u64 obj, u64* zs, u64* p0_out_g2) {
  if (n <= 0) return;
  k_mult_offline<<<grid_for((n + 7) / 8), TPB, 0, st>>>(
      xs, ys, n, k01, k02, make_tag(purpose, C_R1), make_tag(purpose, C_R2),
      make_tag(purpose, C_G1), obj, zs, p0_out_g2);
}

void launch_mult_online_p(cudaStream_t st, const u64* xs, const u64* ys, long long n, Key k01,
                          u32 purpose, u64 obj, const u64* p2_in_g2, u64* p1_out, u64* p2_out) {
  if (n <= 0) return;
  k_mult_online<<<grid_for((n + 7) / 8), TPB, 0, st>>>(xs, ys, n, k01, make_tag(purpose, C_G1),
                                                       obj, p2_in_g2, p1_out, p2_out);
}

void launch_mult_online(cudaStream_t st, const u64* xs, const u64* ys, long long n, Key k01,
                        u64 obj, const u64* p2_in_g2, u64* p1_out, u64* p2_out) {
  if (n <= 0) return;
  k_mult_online<<<grid_for((n + 7) / 8), TPB, 0, st>>>(xs, ys, n, k01, make_tag(P_MULT, C_G1),
                                                       obj, p2_in_g2, p1_out, p2_out);
}

void launch_exchange_finish(cudaStream_t st, long long n, const u64* p1_own, const u64* p1_in,
                            const u64* p2_own, const u64* p2_in, u64* zs, int t, u64* outs) {
  if (n <= 0) return;
  k_exchange_finish<<<grid_for(n), TPB, 0, st>>>(n, p1_own, p1_in, p2_own, p2_in, zs, t, outs);
}

void launch_trunc_p0(cudaStream_t st, long long E, Key k01, Key k02, u64 obj, int t, u64* zpre,
                     u64* zout, u64* pq, u64* p0_out_gp2, u64* p0_out_gq2, u64* p1_out_mp,
                     u64* p1_out_mq, const u64* row_keys, long long N) {
  if (E <= 0) return;
  k_trunc_p0<<<grid_for((E + 7) / 8), TPB, 0, st>>>(
      E, k01, k02, obj, row_keys, N, t, make_tag(P_TRUNC_BITS, C_TB1), make_tag(P_TRUNC_BITS, C_TB2),
      make_tag(P_TRUNC_P, C_R1), make_tag(P_TRUNC_P, C_R2), make_tag(P_TRUNC_P, C_G1),
      make_tag(P_TRUNC_Q, C_R1), make_tag(P_TRUNC_Q, C_R2), make_tag(P_TRUNC_Q, C_G1), zpre, zout,
      pq, p0_out_gp2, p0_out_gq2, p1_out_mp, p1_out_mq);
}

void launch_trunc_finish(cudaStream_t st, long long E, Key k01, Key k02, u64 obj, int t,
                         const u64* p1_in_mp, const u64* p1_in_mq, const u64* p2_in_mp,
                         const u64* p2_in_mq, const u64* p2_gp2, const u64* p2_gq2,
                         const u64* p1_mp1, const u64* p1_mq1, u64* zpre, u64* zout, u64* pq,
                         const u64* row_keys, long long N) {
  if (E <= 0) return;
  k_trunc_finish<<<grid_for((E + 7) / 8), TPB, 0, st>>>(
      E, k01, k02, obj, row_keys, N, t, make_tag(P_TRUNC_BITS, C_TB1), make_tag(P_TRUNC_BITS, C_TB2), p1_in_mp,
      p1_in_mq, p2_in_mp, p2_in_mq, p2_gp2, p2_gq2, p1_mp1, p1_mq1, zpre, zout, pq);
}

void launch_xor_one(cudaStream_t st, u64* p, u64 mask) { k_xor_one<<<1, 1, 0, st>>>(p, mask); }

void launch_prf_words_keyed(cudaStream_t st, long long n, Key key, u32 tag, const u64* row_keys,
                            long long N, u64* out, long long off) {
  if (n <= 0 || off < 0) return;
  k_prf_words_keyed<<<grid_for(n), TPB, 0, st>>>(n, off, key, tag, row_keys, N, out);
}

void launch_prf_words(cudaStream_t st, long long n, Key key, u32 tag, u64 obj, u64* out,
                      long long off) {
  if (n <= 0 || off < 0) return;
  k_prf_words<<<grid_for((off + n + 7) / 8 - off / 8), TPB, 0, st>>>(n, off, key, tag, obj, out);
}

void launch_open_p1(cudaStream_t st, const u64* m, const u64* r1, const u64* r2, long long n,
                    u64* out) {
  if (n <= 0) return;
  k_open_p1<<<grid_for(n), TPB, 0, st>>>(m, r1, r2, n, out);
}

}  // namespace mpc3
