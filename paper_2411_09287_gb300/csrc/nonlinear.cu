// Kernels of the non-linear layers (Sec. 4.3): Boolean <.>^1 sharings over Z_2 stored bit-sliced
// (64 elements per u64 word, planes of n_pad / 64 words), AND gates (Pi_Mult over Z_2), the pieces
// of daBits / edaBits / the MSB carry circuit / B2A, and the GF(2^64) = GR(2, 64) arithmetic of
// the AND-gate verification (an element is one word, bit c = coefficient of x^c, modulus
// f = x^64 + x^4 + x^3 + x + 1).
//
// Layouts.  A Boolean sharing of nw words is 6 nw words, component c at [c nw, (c+1) nw) in the
// order P0.[r]_1, P0.[r]_2, P1.m, P1.[r]_1, P2.m, P2.[r]_2 (as for arithmetic sharings).  A
// Boolean stream's bit i is bit i % 64 of ChaCha20 word i / 64, so word w of a bit-sliced
// operand is stream word w.
#include "kernels.h"

namespace mpc3 {

namespace {

constexpr int TPB = 256;
inline unsigned grid_for(long long n) {
  long long g = (n + TPB - 1) / TPB;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)g;
}
#define GRID_STRIDE(i, n) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// ---- AND gates (Fig. MultP over Z_2: + and - are XOR, products are AND) ------------------------
__global__ void k_and_offline(const u64* __restrict__ xs, const u64* __restrict__ ys, long long nw,
                              Key k01, Key k02, u32 tr1, u32 tr2, u32 tg1, u64 obj,
                              u64* __restrict__ zs, u64* __restrict__ g2_out) {
  GRID_STRIDE(i, nw) {
    const u64 r1 = prf_word(k01, tr1, obj, (u64)i);
    const u64 r2 = prf_word(k02, tr2, obj, (u64)i);
    const u64 g1 = prf_word(k01, tg1, obj, (u64)i);
    const u64 rx = xs[i] ^ xs[nw + i];
    const u64 ry = ys[i] ^ ys[nw + i];
    g2_out[i] = (rx & ry) ^ r1 ^ r2 ^ g1;   // [Gamma]_2 = Gamma - [Gamma]_1, P0 -> P2
    zs[i] = r1;
    zs[nw + i] = r2;
    zs[3 * nw + i] = r1;
    zs[5 * nw + i] = r2;
  }
}

__global__ void k_and_online(const u64* __restrict__ xs, const u64* __restrict__ ys, long long nw,
                             Key k01, u32 tg1, u64 obj, const u64* __restrict__ g2_in,
                             u64* __restrict__ p1_out, u64* __restrict__ p2_out) {
  GRID_STRIDE(i, nw) {
    const u64 g1 = prf_word(k01, tg1, obj, (u64)i);
    p1_out[i] = (xs[2 * nw + i] & ys[3 * nw + i]) ^ (ys[2 * nw + i] & xs[3 * nw + i]) ^ g1;
    const u64 mx = xs[4 * nw + i], my = ys[4 * nw + i];
    p2_out[i] = (mx & my) ^ (mx & ys[5 * nw + i]) ^ (my & xs[5 * nw + i]) ^ g2_in[i];
  }
}

__global__ void k_xor_finish(long long nw, const u64* __restrict__ p1_own, const u64* __restrict__ p1_in,
                             const u64* __restrict__ p2_own, const u64* __restrict__ p2_in,
                             u64* __restrict__ zs) {
  GRID_STRIDE(i, nw) {
    zs[2 * nw + i] = p1_own[i] ^ p1_in[i];
    zs[4 * nw + i] = p2_own[i] ^ p2_in[i];
  }
}

// ---- bits <-> arithmetic sharings ---------------------------------------------------------------
// out (6 n arithmetic words) = the sharing of the n bits: kind 0 (eta01 bits): [r]_1 = -b;
// kind 1 (eta02 bits): [r]_2 = -b; kind 2 (eta12 bits): m = b (reading A1).
__global__ void k_bits_to_arith(const u64* __restrict__ bits, long long n, int kind, u64* __restrict__ out) {
  GRID_STRIDE(i, n) {
    const u64 b = (bits[i >> 6] >> (i & 63)) & 1ull;
    const u64 nb = 0ull - b;
    out[i] = kind == 0 ? nb : 0ull;
    out[n + i] = kind == 1 ? nb : 0ull;
    out[2 * n + i] = kind == 2 ? b : 0ull;
    out[3 * n + i] = kind == 0 ? nb : 0ull;
    out[4 * n + i] = kind == 2 ? b : 0ull;
    out[5 * n + i] = kind == 1 ? nb : 0ull;
  }
}

// out = a + b - 2 c over all words (linear combination of sharings)
__global__ void k_lin_apb_m2c(long long n, const u64* __restrict__ a, const u64* __restrict__ b,
                              const u64* __restrict__ c, u64* __restrict__ out) {
  GRID_STRIDE(i, n) { out[i] = a[i] + b[i] - 2ull * c[i]; }
}

// ---- edaBit inner products: z_e = sum_i m_{i,e} (2^(i+1) r'_{i,e}), plane-major inputs ---------
// X = <m_i> (only m components non-zero), Y = r' (all components); Pi_Inner (Fig. DPP) per e.
// P0's part: Gamma_e = sum_i r_{x,i} r_{y,i} + [r_z]_1 + [r_z]_2 with r_x = [r]_1 + [r]_2 = 0 for
// every <m_i> (an eta12 bit has no mask), so Gamma_e is the output mask itself.
__global__ void k_eda_inner_offline(long long np, Key k01, Key k02, u32 tr1, u32 tr2, u32 tg1,
                                    u64 obj, u64* __restrict__ zs, u64* __restrict__ g2_out) {
  GRID_STRIDE(e, np) {
    const u64 r1 = prf_word(k01, tr1, obj, (u64)e);
    const u64 r2 = prf_word(k02, tr2, obj, (u64)e);
    const u64 g1 = prf_word(k01, tg1, obj, (u64)e);
    g2_out[e] = r1 + r2 - g1;
    zs[e] = r1;
    zs[np + e] = r2;
    zs[3 * np + e] = r1;
    zs[5 * np + e] = r2;
  }
}

__device__ __forceinline__ u64 shl_mod(u64 v, int s) { return s < 64 ? v << s : 0ull; }

__global__ void k_eda_inner_online(const u64* __restrict__ mbits, const u64* __restrict__ rp,
                                   long long np, Key k01, u32 tg1, u64 obj,
                                   const u64* __restrict__ g2_in, u64* __restrict__ p1_out,
                                   u64* __restrict__ p2_out) {
  const long long N = 64 * np;
  GRID_STRIDE(e, np) {
    u64 s1 = 0, s2 = 0;
    for (int i = 0; i < 64; ++i) {
      const long long j = (long long)i * np + e;
      const u64 m = (mbits[j >> 6] >> (j & 63)) & 1ull;   // m_x of <m_i> (P1 and P2 copies)
      const int sh = i + 1;
      const u64 ry1 = shl_mod(rp[3 * N + j], sh);
      const u64 my2 = shl_mod(rp[4 * N + j], sh), ry2 = shl_mod(rp[5 * N + j], sh);
      // P1: -(m_x [r_y]_1 + m_y [r_x]_1), [r_x]_1 = 0;  P2: m_x m_y - m_x [r_y]_2 - m_y [r_x]_2
      s1 -= m * ry1;
      s2 += m * my2 - m * ry2;
    }
    p1_out[e] = s1 + prf_word(k01, tg1, obj, (u64)e);
    p2_out[e] = s2 + g2_in[e];
  }
}

// ra = sum_i 2^i (<m_i> + <r'_i>) - <z>   (all six components)
__global__ void k_eda_compose(const u64* __restrict__ mbits, const u64* __restrict__ rp,
                              const u64* __restrict__ z, long long np, u64* __restrict__ ra) {
  const long long N = 64 * np;
  GRID_STRIDE(t, 6 * np) {
    const int c = (int)(t / np);
    const long long e = t % np;
    u64 acc = 0;
    for (int i = 0; i < 64; ++i) {
      const long long j = (long long)i * np + e;
      const u64 m = (c == 2 || c == 4) ? (mbits[j >> 6] >> (j & 63)) & 1ull : 0ull;
      acc += (m + rp[c * N + j]) << i;
    }
    ra[c * np + e] = acc - z[c * np + e];
  }
}

// ---- MSB carry circuit ------------------------------------------------------------------------
// Leaves: G_i = r[i] AND Delta_i (all components), P_i = r[i] XOR Delta_i (m components), i < 63;
// leaf 63 = (0, 1).  rbits, G, P: Boolean sharings of 64 planes of W words; dplanes: 64 x W.
__global__ void k_msb_leaves(const u64* __restrict__ rbits, const u64* __restrict__ dplanes, long long W,
                             u64* __restrict__ G, u64* __restrict__ P) {
  const long long NW = 64 * W;
  GRID_STRIDE(t, NW) {
    const int i = (int)(t / W);
    const u64 d = dplanes[t];
    for (int c = 0; c < 6; ++c) {
      const u64 r = rbits[c * NW + t];
      const bool m = (c == 2 || c == 4);
      if (i < 63) {
        G[c * NW + t] = r & d;
        P[c * NW + t] = m ? (r ^ d) : r;
      } else {
        G[c * NW + t] = 0;
        P[c * NW + t] = m ? ~0ull : 0ull;
      }
    }
  }
}

// Level inputs: X = [P_hi(k), k < C ; P_hi(k), k < C (not at the root)],
//               Y = [G_lo(k) ; P_lo(k)], hi = 2k + 1, lo = 2k.  G, P have 2C planes.
__global__ void k_msb_gather(const u64* __restrict__ G, const u64* __restrict__ P, int C, int root,
                             long long W, u64* __restrict__ X, u64* __restrict__ Y) {
  const int planes = root ? C : 2 * C;
  const long long nin = 2ll * C * W, nout = (long long)planes * W;
  GRID_STRIDE(t, nout) {
    const int p = (int)(t / W);
    const long long w = t % W;
    const int k = p < C ? p : p - C;
    for (int c = 0; c < 6; ++c) {
      X[c * nout + t] = P[c * nin + (long long)(2 * k + 1) * W + w];
      Y[c * nout + t] = p < C ? G[c * nin + (long long)(2 * k) * W + w]
                              : P[c * nin + (long long)(2 * k) * W + w];
    }
  }
}

// G'(k) = G_hi(k) XOR Z(k), P'(k) = Z(C + k)
__global__ void k_msb_combine(const u64* __restrict__ G, const u64* __restrict__ Z, int C, int root,
                              long long W, u64* __restrict__ Gout, u64* __restrict__ Pout) {
  const long long nin = 2ll * C * W, nz = (long long)(root ? C : 2 * C) * W, nout = (long long)C * W;
  GRID_STRIDE(t, nout) {
    const int k = (int)(t / W);
    const long long w = t % W;
    for (int c = 0; c < 6; ++c) {
      Gout[c * nout + t] = G[c * nin + (long long)(2 * k + 1) * W + w] ^ Z[c * nz + t];
      if (!root) Pout[c * nout + t] = Z[c * nz + (long long)(C + k) * W + w];
    }
  }
}

// msb = r[63] XOR G_root XOR Delta_63 (public, m components); ge = NOT msb when `negate`.
__global__ void k_msb_out(const u64* __restrict__ rbits, const u64* __restrict__ Groot,
                          const u64* __restrict__ d63, long long W, int negate, u64* __restrict__ out) {
  const long long NW = 64 * W;
  GRID_STRIDE(w, W) {
    for (int c = 0; c < 6; ++c) {
      u64 v = rbits[c * NW + 63 * W + w] ^ Groot[c * W + w];
      if (c == 2 || c == 4) v ^= d63[w] ^ (negate ? ~0ull : 0ull);
      out[c * W + w] = v;
    }
  }
}

// Boolean XOR of two sharings of nw words (6 nw words each)
__global__ void k_bxor(long long n6, const u64* __restrict__ a, const u64* __restrict__ b, u64* __restrict__ out) {
  GRID_STRIDE(i, n6) { out[i] = a[i] ^ b[i]; }
}

// B2A: out = Delta + (1 - 2 Delta) ra for public bits Delta (n elements, packed)
__global__ void k_b2a_apply(const u64* __restrict__ dbits, const u64* __restrict__ ra, long long n,
                            u64* __restrict__ out) {
  GRID_STRIDE(t, 6 * n) {
    const int c = (int)(t / n);
    const long long e = t % n;
    const u64 d = (dbits[e >> 6] >> (e & 63)) & 1ull;
    u64 v = d ? 0ull - ra[t] : ra[t];
    if (d && (c == 2 || c == 4)) v += 1ull;
    out[t] = v;
  }
}

// ---- GF(2^64) ------------------------------------------------------------------------------
// 32 x 32 -> 64-bit carry-less product from integer multiplies on bits spaced 4 apart (the
// "multiplication with holes" of T. Pornin's constant-time GHASH): with x_k = x & (0x11111111 << k),
// the integer product x_i y_j has partial-product bits only in the columns p = i + j (mod 4),
// at most 8 in a column, so each column count fits in the 4 bits p .. p + 3 and bit p is its
// parity.  The XOR of the four products with i + j = k (mod 4), kept at those columns, gives the
// carry-less product's bits there.
__host__ __device__ __forceinline__ u64 clmul32(unsigned x, unsigned y) {
  const unsigned m = 0x11111111u;
  const unsigned x0 = x & m, x1 = x & (m << 1), x2 = x & (m << 2), x3 = x & (m << 3);
  const unsigned y0 = y & m, y1 = y & (m << 1), y2 = y & (m << 2), y3 = y & (m << 3);
  auto mw = [](unsigned a, unsigned b) { return (u64)a * (u64)b; };
  const u64 z0 = mw(x0, y0) ^ mw(x1, y3) ^ mw(x2, y2) ^ mw(x3, y1);
  const u64 z1 = mw(x0, y1) ^ mw(x1, y0) ^ mw(x2, y3) ^ mw(x3, y2);
  const u64 z2 = mw(x0, y2) ^ mw(x1, y1) ^ mw(x2, y0) ^ mw(x3, y3);
  const u64 z3 = mw(x0, y3) ^ mw(x1, y2) ^ mw(x2, y1) ^ mw(x3, y0);
  const u64 M = 0x1111111111111111ull;
  return (z0 & M) | (z1 & (M << 1)) | (z2 & (M << 2)) | (z3 & (M << 3));
}

// a b in GF(2^64) = GF(2)[x] / (x^64 + x^4 + x^3 + x + 1): the 128-bit carry-less product by one
// Karatsuba step over 32-bit halves, then the reduction
__host__ __device__ __forceinline__ u64 gf_mul(u64 a, u64 b) {
  const unsigned a0 = (unsigned)a, a1 = (unsigned)(a >> 32);
  const unsigned b0 = (unsigned)b, b1 = (unsigned)(b >> 32);
  const u64 l = clmul32(a0, b0), h = clmul32(a1, b1);
  const u64 mid = clmul32(a0 ^ a1, b0 ^ b1) ^ l ^ h;
  u64 lo = l ^ (mid << 32);
  const u64 hi = h ^ (mid >> 32);
  // x^64 = x^4 + x^3 + x + 1: fold hi twice (the second fold has at most 4 bits)
  const u64 h2 = (hi >> 60) ^ (hi >> 61) ^ (hi >> 63);
  lo ^= hi ^ (hi << 1) ^ (hi << 3) ^ (hi << 4);
  lo ^= h2 ^ (h2 << 1) ^ (h2 << 3) ^ (h2 << 4);
  return lo;
}

__host__ __device__ u64 gf_pow(u64 a, unsigned long long e) {
  u64 r = 1;
  while (e) {
    if (e & 1) r = gf_mul(r, a);
    a = gf_mul(a, a);
    e >>= 1;
  }
  return r;
}

__host__ __device__ __forceinline__ u64 gf_inv(u64 a) { return gf_pow(a, ~0ull - 1ull); }   // a^(2^64 - 2)

// out[i] = r^i for i < n: each thread computes 64 consecutive powers
__global__ void k_gf_powers(const u64* __restrict__ rp, long long n, u64* __restrict__ out) {
  const u64 r = *rp;
  GRID_STRIDE(b, (n + 63) / 64) {
    u64 p = gf_pow(r, (unsigned long long)(b * 64));
    for (int j = 0; j < 64; ++j) {
      const long long i = b * 64 + j;
      if (i >= n) break;
      out[i] = p;
      p = gf_mul(p, r);
    }
  }
}

// Pi_Tran of AND triples (bits): x'_i = X_i r^i, y'_i = Y_i (lifted), z = sum_i Z_i r^i, per
// component; X, Y, Z: 6 x nw words (bit i of the flattened triples = bit i % 64 of word i / 64).
__global__ void k_gf_tran(const u64* __restrict__ X, const u64* __restrict__ Y, const u64* __restrict__ Z,
                          long long nw, const u64* __restrict__ pw, long long ld, u64* __restrict__ xo,
                          u64* __restrict__ yo, u64* __restrict__ zsum) {
  const long long D = 64 * nw;
  __shared__ u64 red[6][TPB];
  u64 zl[6] = {0, 0, 0, 0, 0, 0};
  GRID_STRIDE(i, D) {
    const u64 p = pw[i];
    const long long w = i >> 6;
    const int b = (int)(i & 63);
    for (int c = 0; c < 6; ++c) {
      xo[c * ld + i] = ((X[c * nw + w] >> b) & 1ull) ? p : 0ull;
      yo[c * ld + i] = (Y[c * nw + w] >> b) & 1ull;
      zl[c] ^= ((Z[c * nw + w] >> b) & 1ull) ? p : 0ull;
    }
  }
  for (int c = 0; c < 6; ++c) red[c][threadIdx.x] = zl[c];
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 6; ++c) red[c][threadIdx.x] ^= red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 6)
    atomicXor(reinterpret_cast<unsigned long long*>(zsum + threadIdx.x),
              (unsigned long long)red[threadIdx.x][0]);
}

// Party sums of a secure GF inner product sum_i u_i v_i over the first D elements (components
// may be absent: null):  S[0] = sum r_u r_v (P0), S[1] = sum (m_u [r_v]_1 + m_v [r_u]_1) (P1),
// S[2] = sum (m_u m_v + m_u [r_v]_2 + m_v [r_u]_2) (P2) (over Z_2 the signs vanish).  XOR-added
// into S; with fold set, u (and v) are given as a fold of two halves: u_i = fa u_{2i} +
// fb u_{2i+1}, i < D (fold = 2: fa = 1 + x, fb = x, taken as a shift and an XOR).
struct GfVec {
  const u64* c[6];
};
__device__ __forceinline__ u64 gv(const GfVec& v, int c, long long i) { return v.c[c] ? v.c[c][i] : 0ull; }
// a x in GF(2^64): a shift, and x^4 + x^3 + x + 1 for the x^64 that it carries out
__device__ __forceinline__ u64 gf_mulx(u64 a) { return (a << 1) ^ ((0ull - (a >> 63)) & 0x1Bull); }
// fold = 1: fa a_{2i} + fb a_{2i+1}; fold = 2: the same at fa = 1 + x, fb = x, which is
// a_{2i} + x (a_{2i} + a_{2i+1})
__device__ __forceinline__ u64 gvf(const GfVec& v, int c, long long i, int fold, u64 fa, u64 fb) {
  if (!v.c[c]) return 0ull;
  if (!fold) return v.c[c][i];
  const u64 a = v.c[c][2 * i], b = v.c[c][2 * i + 1];
  if (fold == 2) return a ^ gf_mulx(a ^ b);
  return gf_mul(fa, a) ^ gf_mul(fb, b);
}

__global__ void k_gf_party_sums(GfVec u, GfVec v, long long D, long long stride, long long off,
                                int fold, u64 fa, u64 fb, u64* __restrict__ S) {
  __shared__ u64 red[3][TPB];
  u64 s0 = 0, s1 = 0, s2 = 0;
  GRID_STRIDE(t, D) {
    const long long i = fold ? t : t * stride + off;
    const u64 ur1 = gvf(u, 0, i, fold, fa, fb) ^ gvf(u, 1, i, fold, fa, fb);
    const u64 vr1 = gvf(v, 0, i, fold, fa, fb) ^ gvf(v, 1, i, fold, fa, fb);
    s0 ^= gf_mul(ur1, vr1);
    s1 ^= gf_mul(gvf(u, 2, i, fold, fa, fb), gvf(v, 3, i, fold, fa, fb)) ^
          gf_mul(gvf(v, 2, i, fold, fa, fb), gvf(u, 3, i, fold, fa, fb));
    const u64 mu = gvf(u, 4, i, fold, fa, fb), mv = gvf(v, 4, i, fold, fa, fb);
    s2 ^= gf_mul(mu, mv) ^ gf_mul(mu, gvf(v, 5, i, fold, fa, fb)) ^ gf_mul(mv, gvf(u, 5, i, fold, fa, fb));
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  red[2][threadIdx.x] = s2;
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] ^= red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 3)
    atomicXor(reinterpret_cast<unsigned long long*>(S + threadIdx.x), (unsigned long long)red[threadIdx.x][0]);
}

// out_i = (1 + zeta) v_{2i} + zeta v_{2i+1} (the fold f(zeta) = (1 - zeta) f(0) + zeta f(1)),
// i < Dh; v has D elements (v_D = 0 when D is odd).  grid.y = 12 folds the six components of
// two vectors: q = blockIdx.y takes component q / 2 of x (q even) or y (q odd), component c at
// c * cap of the input and c * ocap of the output.
__global__ void k_gf_fold(const u64* __restrict__ xv, const u64* __restrict__ yv, long long cap,
                          long long D, const u64* __restrict__ zp, u64* __restrict__ xo,
                          u64* __restrict__ yo, long long ocap) {
  const int q = blockIdx.y;
  const u64* __restrict__ v = ((q & 1) ? yv : xv) + (q >> 1) * cap;
  u64* __restrict__ out = ((q & 1) ? yo : xo) + (q >> 1) * ocap;
  const u64 z = *zp, z1 = z ^ 1ull;
  const long long Dh = (D + 1) / 2;
  GRID_STRIDE(i, Dh) {
    const u64 a = v[2 * i];
    const u64 b = (2 * i + 1 < D) ? v[2 * i + 1] : 0ull;
    out[i] = gf_mul(z1, a) ^ gf_mul(z, b);
  }
}

// Finish of a secure GF inner product (Fig. DPP over GF(2^64)) from the party sums S[0..2]:
// masks [r_h]_1, [r_h]_2 and [Gamma]_1 are word 0 of the (purpose, obj) streams.
__global__ void k_gf_inner_finish(const u64* __restrict__ S, Key k01, Key k02, u32 t1, u32 t2,
                                  u32 tg, u64 obj, u64* __restrict__ h6) {
  const u64 r1 = prf_word(k01, t1, obj, 0);
  const u64 r2 = prf_word(k02, t2, obj, 0);
  const u64 g1 = prf_word(k01, tg, obj, 0);
  const u64 g2 = S[0] ^ r1 ^ r2 ^ g1;   // P0 -> P2
  const u64 m1 = S[1] ^ g1;             // P1
  const u64 m2 = S[2] ^ g2;             // P2
  h6[0] = r1;
  h6[1] = r2;
  h6[2] = m1 ^ m2;
  h6[3] = r1;
  h6[4] = m1 ^ m2;
  h6[5] = r2;
}

// A random shared GF element (r1, r2, m from the three pair streams, word 0) and its Pi_Rec
// (hashes of one word each; a mismatch sets `flag`); out = m + [r]_1 + [r]_2.
__device__ void sha256_word(u64 w, u32 h[8]) {
  u32 blk[16];
  sha256_init(h);
  blk[0] = bswap32((u32)w);
  blk[1] = bswap32((u32)(w >> 32));
  blk[2] = 0x80000000u;
  for (int q = 3; q < 15; ++q) blk[q] = 0;
  blk[15] = 64u;
  sha256_compress(h, blk);
}

__global__ void k_gf_random_shared(Key k01, Key k02, Key k12, u32 t1, u32 t2, u32 tm, u64 obj,
                                   u64* __restrict__ s6) {
  const u64 r1 = prf_word(k01, t1, obj, 0);
  const u64 r2 = prf_word(k02, t2, obj, 0);
  const u64 m = prf_word(k12, tm, obj, 0);
  s6[0] = r1;
  s6[1] = r2;
  s6[2] = m;
  s6[3] = r1;
  s6[4] = m;
  s6[5] = r2;
}

__global__ void k_gf_rec1(const u64* __restrict__ s6, u64 xor_mask, u64* __restrict__ out,
                          u32* status, u32 flag) {
  // 6 threads: one hash each (sent and received copies of the three messages)
  __shared__ u32 dig[6][8];
  const int t = threadIdx.x;
  const u64 in_p1_r2 = s6[1] ^ xor_mask;
  if (t < 6) {
    const u64 v = t == 0 ? s6[3]      // P1: H([r]_1) -> P2
                : t == 1 ? s6[4]      // P2: H(m) -> P0
                : t == 2 ? s6[5]      // P2: H([r]_2) -> P1
                : t == 3 ? s6[0]      // P2 hashes the [r]_1 it received
                : t == 4 ? s6[2]      // P0 hashes the m it received
                         : in_p1_r2;  // P1 hashes the [r]_2 it received
    sha256_word(v, dig[t]);
  }
  __syncthreads();
  if (t < 8 && (dig[0][t] != dig[3][t] || dig[1][t] != dig[4][t] || dig[2][t] != dig[5][t]))
    atomicOr(status, flag);
  if (t == 0) *out = s6[2] ^ s6[3] ^ in_p1_r2;   // P1's opening
}

// Lagrange weights at the points 0, 1, x (reading A6/X) over GF(2^64):
// L0 = (z - 1)(z - x) / x, L1 = z (z - x) / (1 - x), L2 = z (z - 1) / (x (x - 1)).
// coef: [0] zeta, [1] L0, [2] L1, [3] L2, [4] 1 + x (the fold weight of f(0) at the point x).
// The three denominators are constants: their inverses (inv[0..2]) come from the host.
struct GfLagInv {
  u64 v[3];
};
__global__ void k_gf_lagrange(const u64* __restrict__ zp, u64* __restrict__ coef, GfLagInv inv) {
  const u64 z = *zp, x = 2ull, one = 1ull;
  coef[0] = z;
  coef[1] = gf_mul(gf_mul(z ^ one, z ^ x), inv.v[0]);
  coef[2] = gf_mul(gf_mul(z, z ^ x), inv.v[1]);
  coef[3] = gf_mul(gf_mul(z, z ^ one), inv.v[2]);
  coef[4] = one ^ x;
}

// z_new = L0 h0 + L1 (z - h0) + L2 h2 per component
__global__ void k_gf_combine_z(const u64* __restrict__ coef, const u64* __restrict__ h0,
                               const u64* __restrict__ h2, const u64* __restrict__ z, u64* __restrict__ zo) {
  const int c = threadIdx.x;
  if (c < 6) zo[c] = gf_mul(coef[1], h0[c]) ^ gf_mul(coef[2], z[c] ^ h0[c]) ^ gf_mul(coef[3], h2[c]);
}

// secure x_i * alpha (Fig. MultP over GF(2^64)) for i < D, all components of x present or null:
// offline P0 part (masks, [Gamma]_2 message) and the online parts, fused; messages are counted
// by the caller.  xa: 6 x D words.
__global__ void k_gf_mult_alpha(GfVec x, const u64* __restrict__ a6, long long D, long long ld,
                                Key k01, Key k02, u32 tr1, u32 tr2, u32 tg1, u64 obj,
                                u64* __restrict__ xa) {
  GRID_STRIDE(i, D) {
    const u64 rz1 = prf_word(k01, tr1, obj, (u64)i);
    const u64 rz2 = prf_word(k02, tr2, obj, (u64)i);
    const u64 g1 = prf_word(k01, tg1, obj, (u64)i);
    const u64 rx = gv(x, 0, i) ^ gv(x, 1, i), ra = a6[0] ^ a6[1];
    const u64 g2 = gf_mul(rx, ra) ^ rz1 ^ rz2 ^ g1;
    const u64 m1 = gf_mul(gv(x, 2, i), a6[3]) ^ gf_mul(a6[2], gv(x, 3, i)) ^ g1;
    const u64 mx = gv(x, 4, i), ma = a6[4];
    const u64 m2 = gf_mul(mx, ma) ^ gf_mul(mx, a6[5]) ^ gf_mul(ma, gv(x, 5, i)) ^ g2;
    xa[i] = rz1;
    xa[ld + i] = rz2;
    xa[2 * ld + i] = m1 ^ m2;
    xa[3 * ld + i] = rz1;
    xa[4 * ld + i] = m1 ^ m2;
    xa[5 * ld + i] = rz2;
  }
}

__global__ void k_gf_check_zero(const u64* __restrict__ d, u32* status, u32 flag) {
  if (*d) atomicOr(status, flag);
}

// out = a - b (sub = 1) or a + b (sub = 0) over n words
__global__ void k_addsub(long long n, const u64* __restrict__ a, const u64* __restrict__ b, int sub,
                         u64* __restrict__ out) {
  GRID_STRIDE(i, n) { out[i] = sub ? a[i] - b[i] : a[i] + b[i]; }
}

// P1's opening of a Boolean sharing: m XOR [r]_1 XOR [r]_2 (received)
__global__ void k_open_xor(const u64* __restrict__ m, const u64* __restrict__ r1,
                           const u64* __restrict__ r2_in, long long n, u64* __restrict__ out) {
  GRID_STRIDE(i, n) { out[i] = m[i] ^ r1[i] ^ r2_in[i]; }
}

// Pi_Tran of the edaBit inner products (rows e of dimension 64, weight r^(e0 + e) on row e):
// x'_{(e0+e) 64 + i} = r^(e0+e) <m_i> (components 2 and 4 only: <m_i> has no mask) as GR vectors
// (64 words per entry), and y_{(e0+e) 64 + i} = 2^(i+1) <r'_i> (all components) as ring words, one
// per entry (the lifted vectors' first round reads them as such).
__global__ void k_eda_tran(const u64* __restrict__ mbits, const u64* __restrict__ rp, long long np,
                           const u64* __restrict__ pw, long long e0, u64* __restrict__ x2,
                           u64* __restrict__ x4, u64* const* __restrict__ y) {
  const long long N = 64 * np;
  GRID_STRIDE(t, N * 64) {
    const long long q = t >> 6;            // local entry: e * 64 + i
    const int k = (int)(t & 63);           // GR coefficient
    const long long e = q >> 6;
    const int i = (int)(q & 63);
    const long long j = (long long)i * np + e;
    const long long row = (e0 + e) * 64 + i;
    if (x2) {   // the x vectors (absent when the first round takes them from the bits)
      const u64 m = (mbits[j >> 6] >> (j & 63)) & 1ull;
      const u64 xv = m ? pw[(e0 + e) * 64 + k] : 0ull;
      x2[row * 64 + k] = xv;
      x4[row * 64 + k] = xv;
    }
    if (k < 6) y[k][row] = shl_mod(rp[k * N + j], i + 1);   // component k of the ring word
  }
}

// First Pi_Reduce round of the edaBit inner-product batch without its x vectors: x = r^g <m_i>
// (g = e0 + e the element, i the bit, components 2 and 4, no mask) pairs bits 2k and 2k + 1 of one
// element, so the round's party sums are sum_g r^g s(g) with per-element words s(g) (P0 has none:
// x has no mask), here written to out (6 rows of ld words, element g at column g):
//   rows 0, 1: the even pairs' sums of P1 (-m Y3) and P2 (m (Y4 - Y5)); rows 2, 3: the cross
//   terms; rows 4, 5: the odd pairs'; Y_c = 2^(i+1) <r'_i>_c (the batch's y words).
__global__ void k_eda_r1_sums(const u64* __restrict__ mbits, const u64* __restrict__ rp, long long np,
                              long long e0, long long ld, u64* __restrict__ out) {
  const long long N = 64 * np;
  GRID_STRIDE(e, np) {
    u64 p1[3] = {0, 0, 0}, p2[3] = {0, 0, 0};   // [ee, cross, oo]
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
      const long long ja = (long long)(2 * k) * np + e, jb = ja + np;
      const u64 ma = (mbits[ja >> 6] >> (ja & 63)) & 1ull, mb = (mbits[jb >> 6] >> (jb & 63)) & 1ull;
      const u64 y3a = shl_mod(rp[3 * N + ja], 2 * k + 1), y3b = shl_mod(rp[3 * N + jb], 2 * k + 2);
      const u64 wa = shl_mod(rp[4 * N + ja], 2 * k + 1) - shl_mod(rp[5 * N + ja], 2 * k + 1);
      const u64 wb = shl_mod(rp[4 * N + jb], 2 * k + 2) - shl_mod(rp[5 * N + jb], 2 * k + 2);
      p1[0] += ma * y3a;
      p1[1] += ma * y3b + mb * y3a;
      p1[2] += mb * y3b;
      p2[0] += ma * wa;
      p2[1] += ma * wb + mb * wa;
      p2[2] += mb * wb;
    }
    const long long g = e0 + e;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      out[(2 * b) * ld + g] = 0ull - p1[b];
      out[(2 * b + 1) * ld + g] = p2[b];
    }
  }
}

// The round's x fold without the x vectors: row g 32 + k of the folded vector is
// r^g (m_2k + f (m_2k+1 - m_2k)) = 0, r^g - A_g, A_g or r^g (A_g = r^g f, f the fold element),
// for components 2 and 4.
__global__ void k_eda_x_fold(const u64* __restrict__ mbits, long long np, long long e0,
                             const u64* __restrict__ pw, const u64* __restrict__ A,
                             u64* __restrict__ x2, u64* __restrict__ x4) {
  GRID_STRIDE(t, np * 32 * 64) {
    const int c = (int)(t & 63);
    const long long q = t >> 6;              // local folded row: e * 32 + k
    const long long e = q >> 5;
    const int k = (int)(q & 31);
    const long long ja = (long long)(2 * k) * np + e, jb = ja + np;
    const u64 ma = (mbits[ja >> 6] >> (ja & 63)) & 1ull, mb = (mbits[jb >> 6] >> (jb & 63)) & 1ull;
    const long long g = e0 + e;
    const u64 pv = pw[g * 64 + c], av = A[g * 64 + c];
    const u64 v = ma ? (mb ? pv : pv - av) : (mb ? av : 0ull);
    const long long row = g * 32 + k;
    x2[row * 64 + c] = v;
    x4[row * 64 + c] = v;
  }
}

// 2x2 max-pool operands: for every window w = (b, ch, i, j) of a (B C, H, W) tensor (one
// component of n = B C H W words), left = [a ; c], right = [b ; d] with a = [2i][2j],
// b = [2i][2j+1], c = [2i+1][2j], d = [2i+1][2j+1]; nw windows, stage width np.
__global__ void k_window_gather(const u64* __restrict__ x, long long BC, long long H, long long W,
                                long long np, u64* __restrict__ left, u64* __restrict__ right) {
  const long long H2 = H / 2, W2 = W / 2, nw = BC * H2 * W2, n = BC * H * W;
  GRID_STRIDE(t, 6 * nw) {
    const int c = (int)(t / nw);
    const long long w = t % nw;
    const long long bc = w / (H2 * W2), ij = w % (H2 * W2), i = ij / W2, j = ij % W2;
    const u64* src = x + c * n + (bc * H + 2 * i) * W + 2 * j;
    left[c * np + w] = src[0];
    right[c * np + w] = src[1];
    left[c * np + nw + w] = src[W];
    right[c * np + nw + w] = src[W + 1];
  }
}

// out[c][k] = idx[k] >= 0 ? xs[c][idx[k]] : 0 for the six components (a local linear map)
__global__ void k_gather(const u64* __restrict__ xs, long long n_in, const long long* __restrict__ idx,
                         long long n_out, u64* __restrict__ out) {
  GRID_STRIDE(t, 6 * n_out) {
    const int c = (int)(t / n_out);
    const long long k = t % n_out;
    const long long j = idx[k];
    out[t] = (j >= 0 && j < n_in) ? xs[c * n_in + j] : 0ull;
  }
}

}  // namespace

// ---- launchers ------------------------------------------------------------------------------
void launch_and_offline(cudaStream_t st, const u64* xs, const u64* ys, long long nw, Key k01, Key k02,
                        u32 purpose, u64 obj, u64* zs, u64* g2_out) {
  if (nw <= 0) return;
  k_and_offline<<<grid_for(nw), TPB, 0, st>>>(xs, ys, nw, k01, k02, make_tag(purpose, C_R1),
                                              make_tag(purpose, C_R2), make_tag(purpose, C_G1), obj,
                                              zs, g2_out);
}
void launch_and_online(cudaStream_t st, const u64* xs, const u64* ys, long long nw, Key k01,
                       u32 purpose, u64 obj, const u64* g2_in, u64* p1_out, u64* p2_out) {
  if (nw <= 0) return;
  k_and_online<<<grid_for(nw), TPB, 0, st>>>(xs, ys, nw, k01, make_tag(purpose, C_G1), obj, g2_in,
                                             p1_out, p2_out);
}
void launch_xor_finish(cudaStream_t st, long long nw, const u64* p1_own, const u64* p1_in,
                       const u64* p2_own, const u64* p2_in, u64* zs) {
  if (nw <= 0) return;
  k_xor_finish<<<grid_for(nw), TPB, 0, st>>>(nw, p1_own, p1_in, p2_own, p2_in, zs);
}
void launch_bits_to_arith(cudaStream_t st, const u64* bits, long long n, int kind, u64* out) {
  if (n <= 0) return;
  k_bits_to_arith<<<grid_for(n), TPB, 0, st>>>(bits, n, kind, out);
}
void launch_lin_apb_m2c(cudaStream_t st, long long n, const u64* a, const u64* b, const u64* c, u64* out) {
  if (n <= 0) return;
  k_lin_apb_m2c<<<grid_for(n), TPB, 0, st>>>(n, a, b, c, out);
}
void launch_eda_inner_offline(cudaStream_t st, long long np, Key k01, Key k02, u64 obj, u64* zs,
                              u64* g2_out) {
  k_eda_inner_offline<<<grid_for(np), TPB, 0, st>>>(np, k01, k02, make_tag(P_EDA_INNER, C_R1),
                                                    make_tag(P_EDA_INNER, C_R2),
                                                    make_tag(P_EDA_INNER, C_G1), obj, zs, g2_out);
}
void launch_eda_inner_online(cudaStream_t st, const u64* mbits, const u64* rp, long long np, Key k01,
                             u64 obj, const u64* g2_in, u64* p1_out, u64* p2_out) {
  k_eda_inner_online<<<grid_for(np), TPB, 0, st>>>(mbits, rp, np, k01, make_tag(P_EDA_INNER, C_G1),
                                                   obj, g2_in, p1_out, p2_out);
}
void launch_eda_compose(cudaStream_t st, const u64* mbits, const u64* rp, const u64* z, long long np,
                        u64* ra) {
  k_eda_compose<<<grid_for(6 * np), TPB, 0, st>>>(mbits, rp, z, np, ra);
}
void launch_msb_leaves(cudaStream_t st, const u64* rbits, const u64* dplanes, long long W, u64* G,
                       u64* P) {
  k_msb_leaves<<<grid_for(64 * W), TPB, 0, st>>>(rbits, dplanes, W, G, P);
}
void launch_msb_gather(cudaStream_t st, const u64* G, const u64* P, int C, int root, long long W,
                       u64* X, u64* Y) {
  k_msb_gather<<<grid_for((long long)(root ? C : 2 * C) * W), TPB, 0, st>>>(G, P, C, root, W, X, Y);
}
void launch_msb_combine(cudaStream_t st, const u64* G, const u64* Z, int C, int root, long long W,
                        u64* Gout, u64* Pout) {
  k_msb_combine<<<grid_for((long long)C * W), TPB, 0, st>>>(G, Z, C, root, W, Gout, Pout);
}
void launch_msb_out(cudaStream_t st, const u64* rbits, const u64* Groot, const u64* d63, long long W,
                    int negate, u64* out) {
  k_msb_out<<<grid_for(W), TPB, 0, st>>>(rbits, Groot, d63, W, negate, out);
}
void launch_bxor(cudaStream_t st, long long n6, const u64* a, const u64* b, u64* out) {
  if (n6 <= 0) return;
  k_bxor<<<grid_for(n6), TPB, 0, st>>>(n6, a, b, out);
}
void launch_b2a_apply(cudaStream_t st, const u64* dbits, const u64* ra, long long n, u64* out) {
  k_b2a_apply<<<grid_for(6 * n), TPB, 0, st>>>(dbits, ra, n, out);
}
void launch_gf_powers(cudaStream_t st, const u64* r, long long n, u64* out) {
  if (n <= 0) return;
  k_gf_powers<<<grid_for((n + 63) / 64), TPB, 0, st>>>(r, n, out);
}
void launch_gf_tran(cudaStream_t st, const u64* X, const u64* Y, const u64* Z, long long nw,
                    const u64* pw, long long ld, u64* xo, u64* yo, u64* zsum) {
  if (nw <= 0) return;
  k_gf_tran<<<grid_for(64 * nw), TPB, 0, st>>>(X, Y, Z, nw, pw, ld, xo, yo, zsum);
}
void launch_gf_party_sums(cudaStream_t st, const u64* const u[6], const u64* const v[6], long long D,
                          long long stride, long long off, int fold, u64 fa, u64 fb, u64* S) {
  if (D <= 0) return;
  GfVec U, V;
  for (int c = 0; c < 6; ++c) {
    U.c[c] = u[c];
    V.c[c] = v[c];
  }
  if (fold && fa == 3ull && fb == 2ull) fold = 2;   // the third point x: no general products
  k_gf_party_sums<<<grid_for(D), TPB, 0, st>>>(U, V, D, stride, off, fold, fa, fb, S);
}
void launch_gf_fold6x2(cudaStream_t st, const u64* xv, const u64* yv, long long cap, long long D,
                       const u64* zeta, u64* xo, u64* yo, long long ocap) {
  if (D <= 0) return;
  k_gf_fold<<<dim3(grid_for((D + 1) / 2), 12), TPB, 0, st>>>(xv, yv, cap, D, zeta, xo, yo, ocap);
}
void launch_gf_inner_finish(cudaStream_t st, const u64* S, Key k01, Key k02, u32 purpose, u64 obj,
                            u64* h6) {
  k_gf_inner_finish<<<1, 1, 0, st>>>(S, k01, k02, make_tag(purpose, C_R1), make_tag(purpose, C_R2),
                                     make_tag(purpose, C_G1), obj, h6);
}
void launch_gf_random_shared(cudaStream_t st, Key k01, Key k02, Key k12, u32 purpose, u64 obj,
                             u64* s6) {
  k_gf_random_shared<<<1, 1, 0, st>>>(k01, k02, k12, make_tag(purpose, C_R1),
                                      make_tag(purpose, C_R2), make_tag(purpose, C_M12), obj, s6);
}
void launch_gf_rec1(cudaStream_t st, const u64* s6, u64 xor_mask, u64* out, u32* status, u32 flag) {
  k_gf_rec1<<<1, 32, 0, st>>>(s6, xor_mask, out, status, flag);
}
void launch_gf_lagrange(cudaStream_t st, const u64* zeta, u64* coef) {
  static const GfLagInv inv = [] {
    const u64 x = 2ull, one = 1ull;
    return GfLagInv{{gf_inv(x), gf_inv(one ^ x), gf_inv(gf_mul(x, x ^ one))}};
  }();
  k_gf_lagrange<<<1, 1, 0, st>>>(zeta, coef, inv);
}
void launch_gf_combine_z(cudaStream_t st, const u64* coef, const u64* h0, const u64* h2, const u64* z,
                         u64* zo) {
  k_gf_combine_z<<<1, 32, 0, st>>>(coef, h0, h2, z, zo);
}
void launch_gf_mult_alpha(cudaStream_t st, const u64* const x[6], const u64* a6, long long D,
                          long long ld, Key k01, Key k02, u64 obj, u64* xa) {
  if (D <= 0) return;
  GfVec X;
  for (int c = 0; c < 6; ++c) X.c[c] = x[c];
  k_gf_mult_alpha<<<grid_for(D), TPB, 0, st>>>(X, a6, D, ld, k01, k02, make_tag(P_VER_XA, C_R1),
                                               make_tag(P_VER_XA, C_R2), make_tag(P_VER_XA, C_G1),
                                               obj, xa);
}
void launch_gf_check_zero(cudaStream_t st, const u64* d, u32* status, u32 flag) {
  k_gf_check_zero<<<1, 1, 0, st>>>(d, status, flag);
}

void launch_addsub(cudaStream_t st, long long n, const u64* a, const u64* b, int sub, u64* out) {
  if (n <= 0) return;
  k_addsub<<<grid_for(n), TPB, 0, st>>>(n, a, b, sub, out);
}
void launch_open_xor(cudaStream_t st, const u64* m, const u64* r1, const u64* r2_in, long long n,
                     u64* out) {
  if (n <= 0) return;
  k_open_xor<<<grid_for(n), TPB, 0, st>>>(m, r1, r2_in, n, out);
}
void launch_eda_tran(cudaStream_t st, const u64* mbits, const u64* rp, long long np, const u64* pw,
                     long long e0, u64* x2, u64* x4, u64* const* y_dev) {
  k_eda_tran<<<grid_for(64 * np * 64), TPB, 0, st>>>(mbits, rp, np, pw, e0, x2, x4, y_dev);
}

void launch_eda_r1_sums(cudaStream_t st, const u64* mbits, const u64* rp, long long np, long long e0,
                        long long ld, u64* out) {
  k_eda_r1_sums<<<grid_for(np), TPB, 0, st>>>(mbits, rp, np, e0, ld, out);
}
void launch_eda_x_fold(cudaStream_t st, const u64* mbits, long long np, long long e0, const u64* pw,
                       const u64* A, u64* x2, u64* x4) {
  k_eda_x_fold<<<grid_for(np * 32 * 64), TPB, 0, st>>>(mbits, np, e0, pw, A, x2, x4);
}

void launch_window_gather(cudaStream_t st, const u64* x, long long BC, long long H, long long W,
                          long long np, u64* left, u64* right) {
  k_window_gather<<<grid_for(6 * BC * (H / 2) * (W / 2)), TPB, 0, st>>>(x, BC, H, W, np, left, right);
}

void launch_gather(cudaStream_t st, const u64* xs, long long n_in, const long long* idx,
                   long long n_out, u64* out) {
  if (n_out <= 0) return;
  k_gather<<<grid_for(6 * n_out), TPB, 0, st>>>(xs, n_in, idx, n_out, out);
}

}  // namespace mpc3
