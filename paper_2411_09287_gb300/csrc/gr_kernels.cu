// Kernels on GR(2^64, 64) elements for the batched verification (Sec. 3):
//   random <.>^{l[x]} sharings (Pi_<.>^{l[x]}), powers r^i (Fig. MTP), the Lagrange weights of
//   Pi_Reduce (Fig. Reduce), reduction of Gram sums, the finish of a secure GR inner product
//   (Pi_Inner over GR), the update z' = L0 h(0) + L1 h(1) + L2 h(p2), and the helpers of the
//   truncation-pair batch (weights u_j, the first six reduction rounds evaluated from the matrix
//   S_{j,j'} = sum_e r^(2e) b1_{e,j} b2_{e,j'}, and the materialisation of the folded vectors).
// A GR element is 64 consecutive u64 coefficients.  A <.>^{l[x]}-shared vector of D elements uses
// the 6-component layout with component c at [c*D*64, (c+1)*D*64).
#include "kernels.h"

namespace mpc3 {

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(long long n) {
  long long g = (n + TPB - 1) / TPB;
  if (g > (1ll << 20)) g = 1ll << 20;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// ---- random sharing ---------------------------------------------------------------------------
__global__ void k_gr_random_shared(long long nwords, Key k01, Key k02, Key k12, u32 t1, u32 t2,
                                   u32 tm, u64 obj, u64* __restrict__ s) {
  const long long nb = (nwords + 7) / 8;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
       b += (long long)gridDim.x * blockDim.x) {
    u64 r1[8], r2[8], m[8];
    prf_block8(k01, t1, obj, (u64)b, r1);
    prf_block8(k02, t2, obj, (u64)b, r2);
    prf_block8(k12, tm, obj, (u64)b, m);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long i = b * 8 + j;
      if (i < nwords) {
        s[i] = r1[j];
        s[nwords + i] = r2[j];
        s[2 * nwords + i] = m[j];
        s[3 * nwords + i] = r1[j];
        s[4 * nwords + i] = m[j];
        s[5 * nwords + i] = r2[j];
      }
    }
  }
}

// ---- powers ---------------------------------------------------------------------------------
// Block b writes table[64 b .. 64 b + 63] = a^(64 b) ... ; 64 threads.
__global__ void k_gr_powers(const u64* __restrict__ a, long long n, u64* __restrict__ table) {
  __shared__ u64 acc[64], base[64], av[64], scr[128];
  const int t = threadIdx.x;
  const long long start = (long long)blockIdx.x * 64;
  if (start >= n) return;
  av[t] = a[t];
  base[t] = a[t];
  acc[t] = (t == 0) ? 1ull : 0ull;
  __syncthreads();
  for (long long e = start; e; e >>= 1) {
    if (e & 1) gr_mul_block(acc, base, acc, scr);
    if (e >> 1) gr_mul_block(base, base, base, scr);
  }
  for (int i = 0; i < 64 && start + i < n; ++i) {
    table[(start + i) * 64 + t] = acc[t];
    __syncthreads();
    gr_mul_block(acc, av, acc, scr);
  }
}

__global__ void k_gr_mul1(const u64* a, const u64* b, u64* out) {
  __shared__ u64 sa[64], sb[64], scr[128];
  sa[threadIdx.x] = a[threadIdx.x];
  sb[threadIdx.x] = b[threadIdx.x];
  __syncthreads();
  gr_mul_block(sa, sb, sa, scr);
  out[threadIdx.x] = sa[threadIdx.x];
}

// out = ca * a + cb * b  (single elements; b / cb may be null)
__global__ void k_gr_lincomb(const u64* ca, const u64* a, const u64* cb, const u64* b,
                             u64* out) {
  __shared__ u64 x[64], y[64], s1[64], s2[64], scr[128];
  const int t = threadIdx.x;
  x[t] = a[t];
  s1[t] = ca[t];
  if (b) { y[t] = b[t]; s2[t] = cb[t]; }
  __syncthreads();
  gr_mul_block(s1, x, x, scr);
  if (b) gr_mul_block(s2, y, y, scr);
  out[t] = x[t] + (b ? y[t] : 0ull);
}

// [M_a; M_b]: rows 0..63 the multiplication matrix of a, rows 64..127 that of b.
__global__ void k_gr_mulmat2(const u64* a, const u64* b, u64* M) {
  __shared__ u64 buf[64 * 64];
  const u64* src = (blockIdx.x == 0) ? a : b;
  gr_mulmat_block(src, buf);
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) M[blockIdx.x * 4096 + i] = buf[i];
}

// M[i] = multiplication matrix of the GR element src + i * stride, for i < n (one block each).
__global__ void k_gr_mulmat_batch(const u64* src, long long stride, u64* M) {
  __shared__ u64 buf[64 * 64];
  gr_mulmat_block(src + blockIdx.x * stride, buf);
  u64* dst = M + (long long)blockIdx.x * 4096;
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) dst[i] = buf[i];
}

// out[c * rows + r] = in[r * cols + c] for r < rows, c < cols; entries with r * cols + c >= n
// read as 0 (32 x 32 tiles through shared memory).
__global__ void k_word_transpose(long long rows, long long cols, long long n, const u64* in,
                                 u64* out) {
  __shared__ u64 tile[32][33];
  const long long r0 = (long long)blockIdx.y * 32, c0 = (long long)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 256 threads: 8 rows per pass
  for (int k = ty; k < 32; k += 8) {
    const long long r = r0 + k, c = c0 + tx;
    const long long i = r * cols + c;
    tile[k][tx] = (r < rows && c < cols && i < n) ? in[i] : 0ull;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const long long c = c0 + k, r = r0 + tx;
    if (c < cols && r < rows) out[c * rows + r] = tile[tx][k];
  }
}

// out[i] = src[idx(i)] for rows of 64 words, idx(i) = ((i mul) / div) mod m (m = 0: no mod).
__global__ void k_gather_rows_affine(long long n, const u64* __restrict__ src, long long mul,
                                     long long div, long long m, u64* __restrict__ out) {
  for (long long i = blockIdx.x; i < n; i += gridDim.x) {
    long long idx = (i * mul) / div;
    if (m) idx %= m;
    out[i * 64 + threadIdx.x] = src[idx * 64 + threadIdx.x];
  }
}

// out[c] = sum_{h < nper} in[c nper + h] for c < ncomp (rows of 64 words).
__global__ void k_block_rowsum(long long nper, const u64* __restrict__ in, u64* __restrict__ out) {
  const long long c = blockIdx.x;
  u64 v = 0;
  for (long long h = 0; h < nper; ++h) v += in[(c * nper + h) * 64 + threadIdx.x];
  out[c * 64 + threadIdx.x] = v;
}

// ---- inverses of the interpolation constants (Pi_Reduce with points 0, 1, x) ------------------
__device__ u64 gf2_64_mul(u64 a, u64 b) {   // GF(2)[x]/(x^64 + x^4 + x^3 + x + 1)
  u64 r = 0;
  for (int i = 63; i >= 0; --i) {
    const u64 top = r >> 63;
    r = (r << 1) ^ (top ? 0x1Bull : 0ull);
    if ((b >> i) & 1) r ^= a;
  }
  return r;
}

// out[0..63] = x^-1, out[64..127] = (1 - x)^-1, out[128..191] = (x (x - 1))^-1.
// GF(2^64) inverse a^(2^64 - 2) of the residue, then Newton steps y <- y (2 - a y).
__global__ void k_gr_inverses(u64* out) {
  __shared__ u64 a[64], y[64], t1[64], scr[128];
  __shared__ u64 ybits;
  const int t = threadIdx.x;
  for (int which = 0; which < 3; ++which) {
    // a = x, 1 - x, x^2 - x
    u64 v = 0;
    if (which == 0) v = (t == 1) ? 1ull : 0ull;
    if (which == 1) v = (t == 0) ? 1ull : ((t == 1) ? ~0ull : 0ull);
    if (which == 2) v = (t == 2) ? 1ull : ((t == 1) ? ~0ull : 0ull);
    a[t] = v;
    __syncthreads();
    if (t == 0) {
      u64 bits = 0;
      for (int c = 0; c < 64; ++c) bits |= (a[c] & 1ull) << c;
      u64 acc = 1, p = bits;
      for (int k = 1; k < 64; ++k) {
        p = gf2_64_mul(p, p);
        acc = gf2_64_mul(acc, p);
      }
      ybits = acc;
    }
    __syncthreads();
    y[t] = (ybits >> t) & 1ull;
    __syncthreads();
    for (int it = 0; it < 7; ++it) {
      gr_mul_block(a, y, t1, scr);            // t1 = a y
      t1[t] = ((t == 0) ? 2ull : 0ull) - t1[t];
      __syncthreads();
      gr_mul_block(y, t1, y, scr);            // y = y (2 - a y)
    }
    out[which * 64 + t] = y[t];
    __syncthreads();
  }
}

// ---- Lagrange data of one Pi_Reduce round ---------------------------------------------------
// coef: [0] zeta, [1] L0, [2] L1, [3] L2, [4] 1 - p2, [5] p2, [6] 1 - zeta (64 words each).
__global__ void k_gr_lagrange(const u64* __restrict__ zp, int mode, const u64* __restrict__ inv,
                              u64* __restrict__ coef) {
  __shared__ u64 z[64], a[64], b[64], c[64], scr[128];
  const int t = threadIdx.x;
  const u64 one = (t == 0) ? 1ull : 0ull;
  if (mode == 1) {
    // points 0, 1, 2 at zeta = 2 zeta'
    z[t] = zp[t];
    a[t] = 2 * zp[t] - one;                   // 2z' - 1
    b[t] = zp[t] - one;                       // z' - 1
    __syncthreads();
    gr_mul_block(a, b, c, scr);               // L0 = (2z'-1)(z'-1)
    coef[64 + t] = c[t];
    b[t] = 4 * (one - z[t]);                  // 4 (1 - z')
    __syncthreads();
    gr_mul_block(z, b, c, scr);               // L1 = 4 z' (1 - z')
    coef[128 + t] = c[t];
    gr_mul_block(z, a, c, scr);               // L2 = z' (2z' - 1)
    coef[192 + t] = c[t];
    coef[t] = 2 * z[t];
    coef[256 + t] = ((t == 0) ? ~0ull : 0ull);  // 1 - 2 = -1
    coef[320 + t] = (t == 0) ? 2ull : 0ull;
    coef[384 + t] = one - 2 * z[t];
    return;
  }
  // points 0, 1, x
  const u64 xv = (t == 1) ? 1ull : 0ull;
  z[t] = zp[t];
  a[t] = zp[t] - one;                         // zeta - 1
  b[t] = zp[t] - xv;                          // zeta - x
  __syncthreads();
  gr_mul_block(a, b, c, scr);                 // (zeta-1)(zeta-x)
  a[t] = inv[t];
  __syncthreads();
  gr_mul_block(c, a, c, scr);
  coef[64 + t] = c[t];                        // L0
  gr_mul_block(z, b, c, scr);                 // zeta (zeta - x)
  a[t] = inv[64 + t];
  __syncthreads();
  gr_mul_block(c, a, c, scr);
  coef[128 + t] = c[t];                       // L1
  a[t] = zp[t] - one;
  __syncthreads();
  gr_mul_block(z, a, c, scr);                 // zeta (zeta - 1)
  a[t] = inv[128 + t];
  __syncthreads();
  gr_mul_block(c, a, c, scr);
  coef[192 + t] = c[t];                       // L2
  coef[t] = z[t];
  coef[256 + t] = one - xv;
  coef[320 + t] = xv;
  coef[384 + t] = one - z[t];
}

// ---- fold of Gram sums ------------------------------------------------------------------------
// P: n matrices of 64x64 (P[a][b] = sum u_a v_b); out: n reduced GR elements.
__global__ void k_gr_fold_reduce(const u64* __restrict__ P, u64* __restrict__ out) {
  __shared__ u64 prod[128];
  const u64* M = P + (long long)blockIdx.x * 4096;
  const int s = threadIdx.x;   // 128 threads
  u64 v = 0;
  if (s < 127) {
    const int a0 = (s < 64) ? 0 : s - 63;
    const int a1 = (s < 64) ? s : 63;
    for (int a = a0; a <= a1; ++a) v += M[a * 64 + (s - a)];
  }
  prod[s] = (s < 127) ? v : 0ull;
  __syncthreads();
  if (s < 64) {
    const u64* h = prod + 64;
    u64 r = prod[s] - gr_hg(h, s);
    if (s < 7) {
      u64 h2[3];
      for (int m = 0; m < 3; ++m) h2[m] = gr_hg(h, 64 + m);
      u64 g = 0;
      if (s < 3) g += h2[s];
      if (s - 1 >= 0 && s - 1 < 3) g += h2[s - 1];
      if (s - 3 >= 0 && s - 3 < 3) g += h2[s - 3];
      if (s - 4 >= 0 && s - 4 < 3) g += h2[s - 4];
      r += g;
    }
    out[(long long)blockIdx.x * 64 + s] = r;
  }
}

// ---- secure GR inner product finish -------------------------------------------------------------
// S: [S0 | S1 | S2] reduced party sums: S0 = sum r_u r_v (P0), S1 = -sum(m_u [r_v]_1 + m_v [r_u]_1)
// (P1), S2 = sum(m_u m_v - m_u [r_v]_2 - m_v [r_u]_2) (P2).
// P0: Gamma = S0 + [r_h]_1 + [r_h]_2, sends [Gamma]_2 = Gamma - [Gamma]_1; P1: [m_h]_1 = S1 +
// [Gamma]_1.  Mask components of the output sharing h6 (6 x 64 words) are written here.
__global__ void k_gr_inner_finish1(const u64* __restrict__ S, Key k01, Key k02, u32 t1, u32 t2,
                                   u32 tg, u64 obj, u64* __restrict__ h6,
                                   u64* __restrict__ g2_out, u64* __restrict__ p1_out) {
  const int c = threadIdx.x;   // 64
  const u64 r1 = prf_word(k01, t1, obj, (u64)c);
  const u64 r2 = prf_word(k02, t2, obj, (u64)c);
  const u64 g1 = prf_word(k01, tg, obj, (u64)c);
  h6[c] = r1;
  h6[64 + c] = r2;
  h6[192 + c] = r1;
  h6[320 + c] = r2;
  g2_out[c] = S[c] + r1 + r2 - g1;
  p1_out[c] = S[64 + c] + g1;
}

__global__ void k_gr_inner_finish2(const u64* __restrict__ S, const u64* __restrict__ g2_in,
                                   u64* __restrict__ p2_out) {
  const int c = threadIdx.x;
  p2_out[c] = S[128 + c] + g2_in[c];
}

// z' = L0 h0 + L1 (z - h0) + L2 h2 on each of the 6 components (one block per component).
__global__ void k_gr_combine_z(const u64* __restrict__ coef, const u64* __restrict__ h0,
                               const u64* __restrict__ h2, const u64* __restrict__ z,
                               u64* __restrict__ znew) {
  __shared__ u64 L[64], v[64], acc[64], scr[128];
  const int t = threadIdx.x;
  const int comp = blockIdx.x;
  const long long o = comp * 64;
  L[t] = coef[64 + t];
  v[t] = h0[o + t];
  __syncthreads();
  gr_mul_block(L, v, acc, scr);
  const u64 a0 = acc[t];
  L[t] = coef[128 + t];
  v[t] = z[o + t] - h0[o + t];
  __syncthreads();
  gr_mul_block(L, v, acc, scr);
  const u64 a1 = acc[t];
  L[t] = coef[192 + t];
  v[t] = h2[o + t];
  __syncthreads();
  gr_mul_block(L, v, acc, scr);
  znew[o + t] = a0 + a1 + acc[t];
}

// out[i] = pw[i] * s[i] (GR element times Z_2^64 scalar)
__global__ void k_gr_scale_rows(const u64* __restrict__ pw, const u64* __restrict__ s,
                                long long n, u64* __restrict__ out) {
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < n * 64;
       w += (long long)gridDim.x * blockDim.x)
    out[w] = pw[w] * s[w >> 6];
}

__global__ void k_gr_lift(const u64* __restrict__ s, long long n, u64* __restrict__ out) {
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < n * 64;
       w += (long long)gridDim.x * blockDim.x)
    out[w] = ((w & 63) == 0) ? s[w >> 6] : 0ull;
}

// First Pi_Reduce round of a claim whose y vectors are lifted ring elements (Fig. MTP: y_i = lift
// of a ring word Y_i): the Gram sum G(u, lift(V)) has one non-zero column, so a party sum of the
// round is sum_i V_i u_i, a scalar-weighted sum of GR rows.  For the Dh element pairs of x (rows
// of 64 words) and the words Y (one per element), with A = x0 + x1 and the party terms
//   P0: A (Y0 + Y1),  P1: -(x2 Y3 + x3 Y2),  P2: x4 (Y4 - Y5) - x5 Y4
// (absent components null), adds to S the sums over the pairs of the even elements (ee), the odd
// ones (oo) and the cross terms V_{2i+1} A_{2i} + V_{2i} A_{2i+1} (xo): S[0..2] = ee of P0..P2,
// S[3..5] = xo, S[9..11] = oo, 64 words each.  Element 2 Dh - 1 may be the zero padding: Y
// words past D read as 0.
struct LiftedIn {
  const u64* x[6];
  const u64* y[6];
};
// XM / YM: bit masks of the x and y components that are present (compile-time, so that absent
// components cost neither loads nor registers); XM = YM = 0 reads the masks from the pointers.
template <int XM, int YM>
__global__ void __launch_bounds__(256)
k_gram_lifted(LiftedIn in, long long Dh, long long D, u64* __restrict__ S) {
  const int c = threadIdx.x & 63;       // GR coefficient
  const int slot = threadIdx.x >> 6;    // pair slot of the block (4 per block)
  auto hx = [&](int k) { return XM ? ((XM >> k) & 1) != 0 : in.x[k] != nullptr; };
  auto hy = [&](int k) { return YM ? ((YM >> k) & 1) != 0 : in.y[k] != nullptr; };
  u64 acc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};   // [party][ee, xo, oo]
  for (long long i = (long long)blockIdx.x * 4 + slot; i < Dh; i += (long long)gridDim.x * 4) {
    const long long e0 = 2 * i, e1 = 2 * i + 1;
    u64 xe[6], xo[6], ye[6], yo[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      xe[k] = hx(k) ? in.x[k][e0 * 64 + c] : 0ull;
      xo[k] = hx(k) ? in.x[k][e1 * 64 + c] : 0ull;
      ye[k] = hy(k) ? in.y[k][e0] : 0ull;
      yo[k] = (hy(k) && e1 < D) ? in.y[k][e1] : 0ull;
    }
    const u64 ae = xe[0] + xe[1], ao = xo[0] + xo[1];
    const u64 ve = ye[0] + ye[1], vo = yo[0] + yo[1];
    acc[0][0] += ve * ae;
    acc[0][1] += vo * ae + ve * ao;
    acc[0][2] += vo * ao;
    acc[1][0] -= ye[3] * xe[2] + ye[2] * xe[3];
    acc[1][1] -= yo[3] * xe[2] + ye[3] * xo[2] + yo[2] * xe[3] + ye[2] * xo[3];
    acc[1][2] -= yo[3] * xo[2] + yo[2] * xo[3];
    const u64 we = ye[4] - ye[5], wo = yo[4] - yo[5];
    acc[2][0] += we * xe[4] - ye[4] * xe[5];
    acc[2][1] += wo * xe[4] + we * xo[4] - (yo[4] * xe[5] + ye[4] * xo[5]);
    acc[2][2] += wo * xo[4] - yo[4] * xo[5];
  }
  // the block's 4 slots, then one atomic add per (party, block, coefficient)
  __shared__ u64 red[3][3][4][64];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int b = 0; b < 3; ++b) red[p][b][slot][c] = acc[p][b];
  __syncthreads();
  for (int t = threadIdx.x; t < 9 * 64; t += blockDim.x) {
    const int p = t / 192, b = (t / 64) % 3, cc = t & 63;
    const u64 v = red[p][b][0][cc] + red[p][b][1][cc] + red[p][b][2][cc] + red[p][b][3][cc];
    const int blk = b == 0 ? 0 : (b == 1 ? 3 : 9);   // ee -> S00, xo -> S01, oo -> S11
    atomicAdd(reinterpret_cast<unsigned long long*>(S + (blk + p) * 64 + cc), (unsigned long long)v);
  }
}

// The fold of a lifted y vector: out_i = lift(Y_{2i}) + f (Y_{2i+1} - Y_{2i}) for i < Dh (f: the
// fold's GR element, 64 words; Y words past D read as 0), out rows of 64 words; 16 threads per
// row, 4 coefficients each (16-byte stores).
__global__ void k_fold_lifted(const u64* __restrict__ Y, long long Dh, long long D,
                              const u64* __restrict__ f, u64* __restrict__ out) {
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < Dh * 16;
       w += (long long)gridDim.x * blockDim.x) {
    const long long i = w >> 4;
    const int c = (int)(w & 15) * 4;
    const u64 y0 = Y[2 * i], y1 = 2 * i + 1 < D ? Y[2 * i + 1] : 0ull;
    const u64 d = y1 - y0;
    const ulonglong2 f0 = *reinterpret_cast<const ulonglong2*>(f + c);
    const ulonglong2 f1 = *reinterpret_cast<const ulonglong2*>(f + c + 2);
    ulonglong2* o = reinterpret_cast<ulonglong2*>(out + i * 64 + c);
    o[0] = make_ulonglong2((c == 0 ? y0 : 0ull) + f0.x * d, f0.y * d);
    o[1] = make_ulonglong2(f1.x * d, f1.y * d);
  }
}

__global__ void k_neg_copy(const u64* __restrict__ a, long long n, u64* __restrict__ out) {
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < n;
       w += (long long)gridDim.x * blockDim.x)
    out[w] = 0ull - a[w];
}

__global__ void k_gr_check_zero(const u64* __restrict__ v, u32* status, u32 flag) {
  if (v[threadIdx.x] != 0ull) atomicOr(status, flag);
}

// ---- truncation-pair batch --------------------------------------------------------------------
// u_j = c_j + r c'_j with c_j = -2^(j+1), c'_j = -2 w_j (w_j the weight of bit j in >>_arith t).
__global__ void k_trunc_u(const u64* __restrict__ r, int t, u64* __restrict__ u) {
  const int j = blockIdx.x;
  const int c = threadIdx.x;
  u64 cj = 0ull - (2ull << j);                         // -2^(j+1) mod 2^64 (0 for j = 63)
  if (j == 63) cj = 0;
  u64 wj = 0;
  if (j >= t && j < 63) wj = 1ull << (j - t);
  if (j == 63) {
    wj = (1ull << (63 - t));
    for (int i = 64 - t; i < 64; ++i) wj += 1ull << i;
  }
  const u64 cpj = 0ull - 2 * wj;
  u[j * 64 + c] = r[c] * cpj + ((c == 0) ? cj : 0ull);
}

// P0's sums of one of the first six reduction rounds of the truncation batch (index i = 64 e + j,
// so rounds k = 1..6 fold bits j within one output e).  With V_j, W_j the accumulated public
// weights of the x- and y-side bit j and S_{j,j'} = sum_e r^(2e) b1_{e,j} b2_{e,j'}:
//   h0 = sum_{j, j' in the same 2^(k-1)-block, bit_{k-1}(j) = 0} V_j W_j' S_{j,j'}
//   h2 = sum_{j, j' in the same 2^k-block} lam(j) lam(j') V_j W_j' S_{j,j'},
// lam(j) = lam[0..63] (1 - p2) or lam[64..127] (p2) by bit k-1 of j.  One block per j; results accumulated atomically into
// out[0..63] (h0) and out[64..127] (h2), which must be zero on entry.
__global__ void k_trunc_round_h(const u64* __restrict__ V, const u64* __restrict__ W,
                                const u64* __restrict__ S, int k, const u64* __restrict__ lam,
                                u64* __restrict__ out) {
  __shared__ u64 T0[64], T1[64], a[64], b[64], tmp[64], scr[128];
  const int j = blockIdx.x;
  const int t = threadIdx.x;
  const int sh = k - 1;
  const int blk = 1 << k;
  const int jb = j & ~(blk - 1);
  T0[t] = 0;
  T1[t] = 0;
  __syncthreads();
  for (int jp = jb; jp < jb + blk; ++jp) {
    a[t] = W[jp * 64 + t];
    b[t] = S[((long long)j * 64 + jp) * 64 + t];
    __syncthreads();
    gr_mul_block(a, b, tmp, scr);
    if ((jp >> sh) & 1) T1[t] += tmp[t]; else T0[t] += tmp[t];
    __syncthreads();
  }
  const int aj = (j >> sh) & 1;
  // h0 (only the even half of each 2^k block)
  a[t] = V[j * 64 + t];
  __syncthreads();
  if (aj == 0) {
    gr_mul_block(a, T0, tmp, scr);
    atomicAdd(reinterpret_cast<unsigned long long*>(out + t), tmp[t]);
    __syncthreads();
  }
  // h2: lam(j) V_j (lam0 T0 + lam1 T1)
  b[t] = lam[t];                        // 1 - p2
  __syncthreads();
  gr_mul_block(b, T0, T0, scr);
  b[t] = lam[64 + t];                    // p2
  __syncthreads();
  gr_mul_block(b, T1, T1, scr);
  T0[t] += T1[t];
  __syncthreads();
  gr_mul_block(a, T0, tmp, scr);
  b[t] = lam[aj ? 64 + t : t];
  __syncthreads();
  gr_mul_block(b, tmp, tmp, scr);
  atomicAdd(reinterpret_cast<unsigned long long*>(out + 64 + t), tmp[t]);
}

// After round k: V_j <- w(j) V_j and W_j <- w(j) W_j with w = 1 - zeta or zeta by bit k-1 of j.
__global__ void k_trunc_update_vw(u64* __restrict__ V, u64* __restrict__ W, int k,
                                  const u64* __restrict__ coef) {
  __shared__ u64 a[64], b[64], scr[128];
  const int j = blockIdx.x & 63;
  u64* X = (blockIdx.x < 64) ? V : W;
  const int t = threadIdx.x;
  const int bit = (j >> (k - 1)) & 1;
  a[t] = bit ? coef[t] : coef[384 + t];
  b[t] = X[j * 64 + t];
  __syncthreads();
  gr_mul_block(a, b, b, scr);
  X[j * 64 + t] = b[t];
}

// Materialise a folded truncation-batch vector after kd rounds:
// out[e * (64 >> kd) + jp] = [R_e *] sum_{j >> kd == jp} VW_j * (-bit_j(words[e])).
// 256 threads = 4 groups of 64; group g handles every 4th output, thread t of a group computes
// coefficient t.  The product R_e * X uses one uniform 64-step loop per thread: step i adds
// R_i X_{(t-i) mod 64} to the low coefficient t (i <= t) or to the high coefficient 64 + t
// (i > t), followed by the reduction mod f.  VW in shared memory; R (optional) holds r^(2e).
__global__ void __launch_bounds__(256)
k_trunc_materialize(long long E, const u64* __restrict__ words, const u64* __restrict__ VW,
                    const u64* __restrict__ R, int kd, u64* __restrict__ out) {
  __shared__ u64 vw[64 * 64];
  __shared__ u64 xs[4][64], rr[4][64], hp[4][64];
  const int tid = threadIdx.x;
  const int g = tid >> 6, t = tid & 63;
  for (int i = tid; i < 4096; i += blockDim.x) vw[i] = VW[i];
  __syncthreads();
  const int per = 64 >> kd;
  const int bs = 1 << kd;
  const long long nout = E * per;
  for (long long ob = (long long)blockIdx.x * 4; ob < nout; ob += (long long)gridDim.x * 4) {
    const long long o = ob + g;
    const bool live = o < nout;
    u64 s = 0;
    long long e = 0;
    if (live) {
      e = o / per;
      const int jp = (int)(o % per);
      const u64 w = words[e] >> (jp * bs);
      for (int q = 0; q < bs; ++q)
        if ((w >> q) & 1ull) s -= vw[(jp * bs + q) * 64 + t];
    }
    if (R) {
      xs[g][t] = s;
      rr[g][t] = live ? R[e * 64 + t] : 0ull;
      __syncthreads();
      u64 lo = 0, hi = 0;
#pragma unroll 8
      for (int i = 0; i < 64; ++i) {
        const u64 pr = rr[g][i] * xs[g][(t - i) & 63];
        if (i <= t) lo += pr; else hi += pr;
      }
      hp[g][t] = (t < 63) ? hi : 0ull;   // coefficient 64 + t of the product (t = 63: none)
      __syncthreads();
      const u64* h = hp[g];
      s = lo - gr_hg(h, t);
      if (t < 7) {
        u64 h2[3];
        for (int m = 0; m < 3; ++m) h2[m] = gr_hg(h, 64 + m);
        u64 gg = 0;
        if (t < 3) gg += h2[t];
        if (t - 1 >= 0 && t - 1 < 3) gg += h2[t - 1];
        if (t - 3 >= 0 && t - 3 < 3) gg += h2[t - 3];
        if (t - 4 >= 0 && t - 4 < 3) gg += h2[t - 4];
        s += gg;
      }
    }
    if (live) out[o * 64 + t] = s;
    if (R) __syncthreads();   // xs/rr/hp are rewritten by the next iteration
  }
}


// out[e] = a[e] * b[e] in GR(2^64, 64) for e < n (rows of 64 words; out may alias a or b).
// One warp per element: lane l forms the product coefficients 4l .. 4l + 3 with a sliding window
// over b (zero-padded in shared memory, so no bounds tests), then the warp reduces mod f.  Word j
// of the padded b sits at j + j / 8, which makes the lanes' window loads (4 words apart)
// conflict-free.
__device__ __forceinline__ int padj(int j) { return j + (j >> 3); }

__global__ void __launch_bounds__(256)
k_gr_mul_rows(long long n, const u64* __restrict__ a, const u64* __restrict__ b, u64* out) {
  __shared__ u64 sa[8][64], sbp[8][216], sc[8][128];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int i = l; i < 216; i += 32) sbp[w][i] = 0;
  __syncwarp();
  const long long stride = (long long)gridDim.x * 8;
  for (long long e = (long long)blockIdx.x * 8 + w; e < n; e += stride) {
    sa[w][l] = a[e * 64 + l];
    sa[w][l + 32] = a[e * 64 + l + 32];
    sbp[w][padj(64 + l)] = b[e * 64 + l];
    sbp[w][padj(96 + l)] = b[e * 64 + l + 32];
    __syncwarp();
    const int k0 = 4 * l;
    // window w_m = b[k0 + m - i] = padded word 64 + k0 + m - i
    u64 w0 = sbp[w][padj(64 + k0)], w1 = sbp[w][padj(65 + k0)], w2 = sbp[w][padj(66 + k0)],
        w3 = sbp[w][padj(67 + k0)];
    u64 c0 = 0, c1 = 0, c2 = 0, c3 = 0;
#pragma unroll
    for (int i = 0; i < 64; ++i) {
      const u64 ai = sa[w][i];
      c0 += ai * w0;
      c1 += ai * w1;
      c2 += ai * w2;
      c3 += ai * w3;
      w3 = w2;
      w2 = w1;
      w1 = w0;
      w0 = sbp[w][padj(63 + k0 - i)];
    }
    sc[w][k0] = c0;
    sc[w][k0 + 1] = c1;
    sc[w][k0 + 2] = c2;
    sc[w][k0 + 3] = c3;
    __syncwarp();
    const u64* h = sc[w] + 64;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int t = l + 32 * half;
      u64 v = sc[w][t] - gr_hg(h, t);
      if (t < 7) {
        u64 h2[3];
        for (int m = 0; m < 3; ++m) h2[m] = gr_hg(h, 64 + m);
        u64 g = 0;
        if (t < 3) g += h2[t];
        if (t - 1 >= 0 && t - 1 < 3) g += h2[t - 1];
        if (t - 3 >= 0 && t - 3 < 3) g += h2[t - 3];
        if (t - 4 >= 0 && t - 4 < 3) g += h2[t - 4];
        v += g;
      }
      out[e * 64 + t] = v;
    }
    __syncwarp();
  }
}

// out[c] += sum_{e < n} A[c][e] * R[e] for c < nrows <= 16: GR elements R[e] (rows of 64 words)
// scaled by ring scalars and summed (e.g. sum_e r^(2e) p_c[e] for the truncation batch).  Each
// block takes a contiguous slice of e, 256 e at a time: the slice of A is staged in shared memory
// as [e][c] (a broadcast read per e), and each 64-thread group takes 64 of the 256 e, thread t
// coefficient t of every row c; partial sums are added atomically at the end.
template <int NR>
__global__ void __launch_bounds__(256)
k_scalar_gr_sum(long long n, const u64* __restrict__ A, long long lda, int nrows,
                const u64* __restrict__ R, u64* __restrict__ out) {
  __shared__ __align__(16) u64 as[256][NR];
  const int t = threadIdx.x & 63, grp = threadIdx.x >> 6;
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long e0 = per * blockIdx.x;
  const long long e1 = (e0 + per < n) ? e0 + per : n;
  u64 acc[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = 0;
  for (long long eb = e0; eb < e1; eb += 256) {
    __syncthreads();
    for (int i = threadIdx.x; i < NR * 256; i += 256) {
      const int c = i >> 8, k = i & 255;
      as[k][c] = (c < nrows && eb + k < e1) ? A[c * lda + eb + k] : 0ull;
    }
    __syncthreads();
    const int kmax = (int)((e1 - eb - grp * 64 < 64) ? e1 - eb - grp * 64 : 64);
#pragma unroll 2
    for (int k = 0; k < kmax; ++k) {
      const int kk = grp * 64 + k;
      const u64 r = R[(eb + kk) * 64 + t];
#pragma unroll
      for (int c = 0; c < NR; c += 2) {
        const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(&as[kk][c]);
        acc[c] += w.x * r;
        acc[c + 1] += w.y * r;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NR; ++c)
    if (c < nrows)
      atomicAdd(reinterpret_cast<unsigned long long*>(out + c * 64 + t), (unsigned long long)acc[c]);
}

// ---- fused small steps (single GR elements) -----------------------------------------------
// Pi_Rec of one shared GR element s6 (6 x 64 words): P0 sends [r]_1 to P2 and [r]_2 to P1, P1
// sends m to P0; P1 sends H([r]_1) to P2, P2 sends H(m) to P0 and H([r]_2) to P1.  Each receiver
// hashes what it received and compares; a mismatch sets `flag` in *status.  out = P1's opening
// m - [r]_1 - [r]_2.  (xor_mask, xor_idx) corrupts the P0 -> P1 message (fault site REC_MSG).
__device__ void sha256_words64(const u64* v, u32 h[8]) {   // SHA-256 of 512 bytes
  sha256_init(h);
  u32 blk[16];
  for (int b = 0; b < 8; ++b) {
    for (int q = 0; q < 8; ++q) {
      const u64 w = v[b * 8 + q];
      blk[2 * q] = bswap32((u32)w);
      blk[2 * q + 1] = bswap32((u32)(w >> 32));
    }
    sha256_compress(h, blk);
  }
  for (int q = 0; q < 16; ++q) blk[q] = 0;
  blk[0] = 0x80000000u;
  blk[15] = 4096u;
  sha256_compress(h, blk);
}

__global__ void k_gr_rec1(const u64* __restrict__ s6, u64 xor_mask, int xor_idx,
                          u64* __restrict__ out, u32* status, u32 flag) {
  __shared__ u64 in_p2_r1[64], in_p1_r2[64], in_p0_m[64];
  __shared__ u32 dig[6][8];
  const int t = threadIdx.x;   // 64 threads
  in_p2_r1[t] = s6[t];
  in_p1_r2[t] = s6[64 + t] ^ ((t == xor_idx) ? xor_mask : 0ull);
  in_p0_m[t] = s6[128 + t];
  __syncthreads();
  if (t < 6) {
    const u64* src = (t == 0) ? s6 + 192       // P1: H([r]_1), sent to P2
                   : (t == 1) ? s6 + 256       // P2: H(m), sent to P0
                   : (t == 2) ? s6 + 320       // P2: H([r]_2), sent to P1
                   : (t == 3) ? in_p2_r1       // P2 hashes the [r]_1 it received
                   : (t == 4) ? in_p0_m        // P0 hashes the m it received
                              : in_p1_r2;      // P1 hashes the [r]_2 it received
    sha256_words64(src, dig[t]);
  }
  __syncthreads();
  if (t < 8) {
    if (dig[0][t] != dig[3][t] || dig[1][t] != dig[4][t] || dig[2][t] != dig[5][t])
      atomicOr(status, flag);
  }
  out[t] = s6[128 + t] - s6[192 + t] - in_p1_r2[t];
}

// The whole secure GR inner-product finish for one output element: P0's Gamma and [Gamma]_2
// message, P1's and P2's [m_h]_j and their exchange.  S = [S0 | S1 | S2] party sums.
__global__ void k_gr_inner_finish_all(const u64* __restrict__ S, Key k01, Key k02, u32 t1,
                                      u32 t2, u32 tg, u64 obj, u64* __restrict__ h6) {
  const int c = threadIdx.x;   // 64
  const u64 r1 = prf_word(k01, t1, obj, (u64)c);
  const u64 r2 = prf_word(k02, t2, obj, (u64)c);
  const u64 g1 = prf_word(k01, tg, obj, (u64)c);
  const u64 g2 = S[c] + r1 + r2 - g1;        // P0 -> P2
  const u64 m1 = S[64 + c] + g1;             // P1
  const u64 m2 = S[128 + c] + g2;            // P2 (received g2)
  h6[c] = r1;
  h6[64 + c] = r2;
  h6[128 + c] = m1 + m2;                     // P1: own + received
  h6[192 + c] = r1;
  h6[256 + c] = m1 + m2;                     // P2: received + own
  h6[320 + c] = r2;
}

// out[p] = l00 S00[p] + l01 (S01[p] + S10[p]) + l11 S11[p] for the three parties p, with
// l00 = (1-p2)^2, l01 = (1-p2) p2, l11 = p2^2 (bilinear expansion of h(p2)).
__global__ void k_gr_quad_combine(const u64* __restrict__ lam /*[1-p2 | p2]*/,
                                  const u64* __restrict__ S00, const u64* __restrict__ S01,
                                  const u64* __restrict__ S10, const u64* __restrict__ S11,
                                  u64* __restrict__ out) {
  __shared__ u64 a[64], b[64], l00[64], l01[64], l11[64], v[64], acc[64], scr[128];
  const int t = threadIdx.x;
  const int p = blockIdx.x;
  a[t] = lam[t];
  b[t] = lam[64 + t];
  __syncthreads();
  gr_mul_block(a, a, l00, scr);
  gr_mul_block(a, b, l01, scr);
  gr_mul_block(b, b, l11, scr);
  v[t] = S00[p * 64 + t];
  __syncthreads();
  gr_mul_block(l00, v, acc, scr);
  u64 r = acc[t];
  v[t] = S01[p * 64 + t] + S10[p * 64 + t];
  __syncthreads();
  gr_mul_block(l01, v, acc, scr);
  r += acc[t];
  v[t] = S11[p * 64 + t];
  __syncthreads();
  gr_mul_block(l11, v, acc, scr);
  r += acc[t];
  out[p * 64 + t] = r;
}

// mode constants: cst[0..63] = 1 - p2, [64..127] = p2 (p2 = x, or 2 in the 2*zeta' reading)
__global__ void k_mode_consts(int mode, u64* cst) {
  const int t = threadIdx.x;
  const u64 one = (t == 0) ? 1ull : 0ull;
  const u64 p2 = (mode == 1) ? ((t == 0) ? 2ull : 0ull) : ((t == 1) ? 1ull : 0ull);
  cst[t] = one - p2;
  cst[64 + t] = p2;
}

}  // namespace

// ---- launchers --------------------------------------------------------------------------------
void launch_gr_random_shared(cudaStream_t st, long long n, Key k01, Key k02, Key k12,
                             u32 purpose, u64 obj, u64* s6) {
  const long long nw = n * 64;
  k_gr_random_shared<<<grid_for((nw + 7) / 8), TPB, 0, st>>>(
      nw, k01, k02, k12, make_tag(purpose, C_R1), make_tag(purpose, C_R2),
      make_tag(purpose, C_M12), obj, s6);
}

void launch_gr_powers(cudaStream_t st, const u64* a, long long n, u64* table) {
  if (n <= 0) return;
  k_gr_powers<<<(unsigned)((n + 63) / 64), 64, 0, st>>>(a, n, table);
}

void launch_gr_mul1(cudaStream_t st, const u64* a, const u64* b, u64* out) {
  k_gr_mul1<<<1, 64, 0, st>>>(a, b, out);
}

void launch_gr_lincomb(cudaStream_t st, const u64* ca, const u64* a, const u64* cb, const u64* b,
                       u64* out) {
  k_gr_lincomb<<<1, 64, 0, st>>>(ca, a, cb, b, out);
}

void launch_gr_mulmat2(cudaStream_t st, const u64* a, const u64* b, u64* M) {
  k_gr_mulmat2<<<b ? 2 : 1, 64, 0, st>>>(a, b, M);
}

void launch_gr_mulmat_batch(cudaStream_t st, long long n, const u64* src, long long stride,
                            u64* M) {
  if (n <= 0) return;
  k_gr_mulmat_batch<<<(unsigned)n, 64, 0, st>>>(src, stride, M);
}

void launch_word_transpose(cudaStream_t st, long long rows, long long cols, long long n,
                           const u64* in, u64* out) {
  if (rows <= 0 || cols <= 0) return;
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  k_word_transpose<<<grid, 256, 0, st>>>(rows, cols, n, in, out);
}

void launch_gather_rows_affine(cudaStream_t st, long long n, const u64* src, long long mul,
                               long long div, long long m, u64* out) {
  if (n <= 0) return;
  k_gather_rows_affine<<<(unsigned)(n < 65536 ? n : 65536), 64, 0, st>>>(n, src, mul, div, m, out);
}

void launch_block_rowsum(cudaStream_t st, int ncomp, long long nper, const u64* in, u64* out) {
  if (ncomp <= 0) return;
  k_block_rowsum<<<(unsigned)ncomp, 64, 0, st>>>(nper, in, out);
}

void launch_gr_inverses(cudaStream_t st, u64* out) { k_gr_inverses<<<1, 64, 0, st>>>(out); }

void launch_gr_lagrange(cudaStream_t st, const u64* zeta_prime, int mode, const u64* inv,
                        u64* coef) {
  k_gr_lagrange<<<1, 64, 0, st>>>(zeta_prime, mode, inv, coef);
}

void launch_gr_fold_reduce(cudaStream_t st, const u64* P, int n, u64* out) {
  if (n <= 0) return;
  k_gr_fold_reduce<<<n, 128, 0, st>>>(P, out);
}

void launch_gr_inner_finish1(cudaStream_t st, const u64* S, Key k01, Key k02, u32 purpose,
                             u64 obj, u64* h6, u64* g2_out, u64* p1_out) {
  k_gr_inner_finish1<<<1, 64, 0, st>>>(S, k01, k02, make_tag(purpose, C_R1),
                                       make_tag(purpose, C_R2), make_tag(purpose, C_G1), obj, h6,
                                       g2_out, p1_out);
}

void launch_gr_inner_finish2(cudaStream_t st, const u64* S, const u64* g2_in, u64* p2_out) {
  k_gr_inner_finish2<<<1, 64, 0, st>>>(S, g2_in, p2_out);
}

void launch_gr_combine_z(cudaStream_t st, const u64* coef, const u64* h0, const u64* h2,
                         const u64* z, u64* znew) {
  k_gr_combine_z<<<6, 64, 0, st>>>(coef, h0, h2, z, znew);
}

void launch_gr_scale_rows(cudaStream_t st, const u64* pw, const u64* s, long long n, u64* out) {
  if (n <= 0) return;
  k_gr_scale_rows<<<grid_for(n * 64), TPB, 0, st>>>(pw, s, n, out);
}

void launch_gr_lift(cudaStream_t st, const u64* s, long long n, u64* out) {
  if (n <= 0) return;
  k_gr_lift<<<grid_for(n * 64), TPB, 0, st>>>(s, n, out);
}

void launch_gram_lifted(cudaStream_t st, const u64* const x[6], const u64* const y[6], long long Dh,
                        long long D, u64* S) {
  if (Dh <= 0) return;
  LiftedIn in;
  for (int k = 0; k < 6; ++k) {
    in.x[k] = x[k];
    in.y[k] = y[k];
  }
  long long g = (Dh + 3) / 4;
  if (g > 152 * 8) g = 152 * 8;
  int xm = 0, ym = 0;
  for (int k = 0; k < 6; ++k) {
    xm |= x[k] ? 1 << k : 0;
    ym |= y[k] ? 1 << k : 0;
  }
  // the component patterns of Pi_MultVerify (all), the edaBit inner products (x: the m
  // components) and the edaBit bit products (x: [r]_1, y: [r]_2); any other takes the general form
  if (xm == 63 && ym == 63) k_gram_lifted<63, 63><<<(unsigned)g, 256, 0, st>>>(in, Dh, D, S);
  else if (xm == 0x14 && ym == 63) k_gram_lifted<0x14, 63><<<(unsigned)g, 256, 0, st>>>(in, Dh, D, S);
  else if (xm == 0x09 && ym == 0x22) k_gram_lifted<0x09, 0x22><<<(unsigned)g, 256, 0, st>>>(in, Dh, D, S);
  else k_gram_lifted<0, 0><<<(unsigned)g, 256, 0, st>>>(in, Dh, D, S);
}

void launch_fold_lifted(cudaStream_t st, const u64* Y, long long Dh, long long D, const u64* f,
                        u64* out) {
  if (Dh <= 0) return;
  k_fold_lifted<<<grid_for(Dh * 16), TPB, 0, st>>>(Y, Dh, D, f, out);
}

void launch_neg_copy(cudaStream_t st, const u64* a, long long n, u64* out) {
  if (n <= 0) return;
  k_neg_copy<<<grid_for(n), TPB, 0, st>>>(a, n, out);
}

void launch_gr_check_zero(cudaStream_t st, const u64* v, u32* status, u32 flag) {
  k_gr_check_zero<<<1, 64, 0, st>>>(v, status, flag);
}

void launch_trunc_u(cudaStream_t st, const u64* r, int t, u64* u) {
  k_trunc_u<<<64, 64, 0, st>>>(r, t, u);
}

void launch_trunc_round_h(cudaStream_t st, const u64* V, const u64* W, const u64* S, int k,
                          const u64* lam, u64* out) {
  k_trunc_round_h<<<64, 64, 0, st>>>(V, W, S, k, lam, out);
}

void launch_trunc_update_vw(cudaStream_t st, u64* V, u64* W, int k, const u64* coef) {
  k_trunc_update_vw<<<128, 64, 0, st>>>(V, W, k, coef);
}

void launch_trunc_materialize(cudaStream_t st, long long E, const u64* words, const u64* VW,
                              const u64* R, int kd, u64* out) {
  if (E <= 0) return;
  long long nout = E * (64 >> kd);
  long long g = (nout + 3) / 4;
  if (g > 152 * 16) g = 152 * 16;
  k_trunc_materialize<<<(unsigned)g, 256, 0, st>>>(E, words, VW, R, kd, out);
}

void launch_gr_rec1(cudaStream_t st, const u64* s6, u64 xor_mask, int xor_idx, u64* out,
                    u32* status, u32 flag) {
  k_gr_rec1<<<1, 64, 0, st>>>(s6, xor_mask, xor_idx, out, status, flag);
}

void launch_gr_inner_finish_all(cudaStream_t st, const u64* S, Key k01, Key k02, u32 purpose,
                                u64 obj, u64* h6) {
  k_gr_inner_finish_all<<<1, 64, 0, st>>>(S, k01, k02, make_tag(purpose, C_R1),
                                          make_tag(purpose, C_R2), make_tag(purpose, C_G1), obj,
                                          h6);
}

void launch_gr_quad_combine(cudaStream_t st, const u64* lam, const u64* S00, const u64* S01,
                            const u64* S10, const u64* S11, u64* out) {
  k_gr_quad_combine<<<3, 64, 0, st>>>(lam, S00, S01, S10, S11, out);
}

void launch_mode_consts(cudaStream_t st, int mode, u64* cst) {
  k_mode_consts<<<1, 64, 0, st>>>(mode, cst);
}

void launch_gr_mul_rows(cudaStream_t st, long long n, const u64* a, const u64* b, u64* out) {
  if (n <= 0) return;
  long long g = (n + 7) / 8;
  if (g > 152 * 8) g = 152 * 8;
  k_gr_mul_rows<<<(unsigned)g, 256, 0, st>>>(n, a, b, out);
}

void launch_scalar_gr_sum(cudaStream_t st, long long n, const u64* A, long long lda, int nrows,
                          const u64* R, u64* out) {
  if (n <= 0 || nrows <= 0) return;
  long long g = (n + 4095) / 4096;
  if (g > 152 * 8) g = 152 * 8;
  if (nrows <= 12)
    k_scalar_gr_sum<12><<<(unsigned)g, 256, 0, st>>>(n, A, lda, nrows, R, out);
  else
    k_scalar_gr_sum<16><<<(unsigned)g, 256, 0, st>>>(n, A, lda, nrows, R, out);
}

}  // namespace mpc3
