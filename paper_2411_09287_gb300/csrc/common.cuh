// Device-side building blocks shared by the kernels of libmpc3:
//   * the pairwise PRG (ChaCha20 block function, RFC 8439 Sec. 2.3) that realises the paper's
//     "P_j and P_k pick random values together with seed eta_{j,k}" (Sec. 2, Secret sharing);
//   * arithmetic in the Galois ring GR(2^64, 64) = Z_2^64[x]/f(x), f = x^64 + x^4 + x^3 + x + 1
//     (Sec. 2 Notation, Sec. 3), used by the batched verification;
//   * SHA-256 (FIPS 180-4), the hash H of Pi_Rec (Sec. 2, verifiable reconstruction).
// All ring arithmetic is on uint64_t, i.e. exactly mod 2^64.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpc3 {

typedef uint64_t u64;
typedef uint32_t u32;

constexpr int GR_D = 64;                 // extension degree d (Sec. 5: d = 64)

// ---------------------------------------------------------------------------------------------
// PRG streams.  Element i of stream (tag, obj) under a pair key is the little-endian u64 made of
// state words 2w, 2w+1 (w = i mod 8) of the ChaCha20 block with counter floor(i/8) and nonce
// words (tag, obj mod 2^32, obj >> 32).
// ---------------------------------------------------------------------------------------------
struct Key {
  u32 k[8];
};

// stream components: which pair key a stream is drawn with
enum Comp : u32 { C_R1 = 1, C_R2 = 2, C_M12 = 3, C_G1 = 4, C_TB1 = 5, C_TB2 = 6 };
// stream purposes
enum Purpose : u32 {
  P_SHARE = 0x01, P_MULT = 0x02, P_INNER = 0x03, P_TRUNC_BITS = 0x04, P_TRUNC_P = 0x05,
  P_TRUNC_Q = 0x06, P_DABIT = 0x07, P_EDABIT = 0x08, P_AND = 0x09, P_EDA_MULT = 0x0A,
  P_EDA_INNER = 0x0B, P_DA_MULT1 = 0x0C, P_DA_MULT2 = 0x0D, P_NL_MULT = 0x0E, P_VER_R = 0x10, P_VER_ZETA = 0x11, P_VER_H0 = 0x12, P_VER_H2 = 0x13,
  P_VER_ALPHA = 0x14, P_VER_XA = 0x15, P_VER_DELTA = 0x16
};
__host__ __device__ inline u32 make_tag(u32 purpose, u32 comp) { return (purpose << 4) | comp; }
__host__ __device__ inline u64 make_obj(u64 call_id, u32 batch, u32 sub) {
  return (call_id << 20) | ((u64)batch << 16) | (u64)sub;
}

__device__ __forceinline__ u32 rotl32(u32 x, int n) { return __funnelshift_l(x, x, n); }

#define MPC3_QR(a, b, c, d)            \
  a += b; d ^= a; d = rotl32(d, 16);   \
  c += d; b ^= c; b = rotl32(b, 12);   \
  a += b; d ^= a; d = rotl32(d, 8);    \
  c += d; b ^= c; b = rotl32(b, 7);

// One ChaCha20 block: out[0..15] = state after 20 rounds plus the input state.
__device__ __forceinline__ void chacha_block(const Key& key, u32 counter, u32 n0, u32 n1, u32 n2,
                                             u32 out[16]) {
  u32 x0 = 0x61707865u, x1 = 0x3320646eu, x2 = 0x79622d32u, x3 = 0x6b206574u;
  u32 x4 = key.k[0], x5 = key.k[1], x6 = key.k[2], x7 = key.k[3];
  u32 x8 = key.k[4], x9 = key.k[5], x10 = key.k[6], x11 = key.k[7];
  u32 x12 = counter, x13 = n0, x14 = n1, x15 = n2;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    MPC3_QR(x0, x4, x8, x12) MPC3_QR(x1, x5, x9, x13) MPC3_QR(x2, x6, x10, x14)
    MPC3_QR(x3, x7, x11, x15) MPC3_QR(x0, x5, x10, x15) MPC3_QR(x1, x6, x11, x12)
    MPC3_QR(x2, x7, x8, x13) MPC3_QR(x3, x4, x9, x14)
  }
  out[0] = x0 + 0x61707865u; out[1] = x1 + 0x3320646eu; out[2] = x2 + 0x79622d32u;
  out[3] = x3 + 0x6b206574u; out[4] = x4 + key.k[0]; out[5] = x5 + key.k[1];
  out[6] = x6 + key.k[2]; out[7] = x7 + key.k[3]; out[8] = x8 + key.k[4];
  out[9] = x9 + key.k[5]; out[10] = x10 + key.k[6]; out[11] = x11 + key.k[7];
  out[12] = x12 + counter; out[13] = x13 + n0; out[14] = x14 + n1; out[15] = x15 + n2;
}

// The 8 u64 words of block `blk` of stream (tag, obj).
__device__ __forceinline__ void prf_block8(const Key& key, u32 tag, u64 obj, u64 blk, u64 w[8]) {
  u32 o[16];
  chacha_block(key, (u32)blk, tag, (u32)obj, (u32)(obj >> 32), o);
#pragma unroll
  for (int i = 0; i < 8; ++i) w[i] = (u64)o[2 * i] | ((u64)o[2 * i + 1] << 32);
}

// Element i of stream (tag, obj): one full block for one word (for scattered use).
__device__ __forceinline__ u64 prf_word(const Key& key, u32 tag, u64 obj, u64 i) {
  u32 o[16];
  chacha_block(key, (u32)(i >> 3), tag, (u32)obj, (u32)(obj >> 32), o);
  const int w = (int)(i & 7);
  // select without dynamic register indexing
  u32 lo = 0, hi = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k == w) { lo = o[2 * k]; hi = o[2 * k + 1]; }
  }
  return (u64)lo | ((u64)hi << 32);
}

// ---------------------------------------------------------------------------------------------
// GR(2^64, 64).  Reduction of a 127-coefficient product p = L + x^64 H, deg H <= 62:
// with g = x^4 + x^3 + x + 1 (so x^64 = -g), H g = A + x^64 H2 with deg A <= 63, deg H2 <= 2,
// and p = L - A + g H2 (since -x^64 H2 = g H2).
// ---------------------------------------------------------------------------------------------
__host__ __device__ inline u64 gr_hg(const u64* h, int s) {   // (H g)_s, h has 63 entries
  u64 v = 0;
  if (s >= 0 && s < 63) v += h[s];
  if (s - 1 >= 0 && s - 1 < 63) v += h[s - 1];
  if (s - 3 >= 0 && s - 3 < 63) v += h[s - 3];
  if (s - 4 >= 0 && s - 4 < 63) v += h[s - 4];
  return v;
}

// Serial reduction (one thread): out[c] for c < 64 from p[0..126].
__host__ __device__ inline void gr_reduce_serial(const u64* p, u64* out) {
  const u64* h = p + 64;
  u64 h2[3];
  for (int m = 0; m < 3; ++m) h2[m] = gr_hg(h, 64 + m);
  for (int c = 0; c < 64; ++c) {
    u64 v = p[c] - gr_hg(h, c);
    if (c < 7) {
      u64 g = 0;
      if (c < 3) g += h2[c];
      if (c - 1 >= 0 && c - 1 < 3) g += h2[c - 1];
      if (c - 3 >= 0 && c - 3 < 3) g += h2[c - 3];
      if (c - 4 >= 0 && c - 4 < 3) g += h2[c - 4];
      v += g;
    }
    out[c] = v;
  }
}

// Block-cooperative product out = a * b (64 threads of the block participate with tid < 64;
// other threads idle).  `scratch` holds 128 words of shared memory.  a, b, out may alias.
__device__ inline void gr_mul_block(const u64* a, const u64* b, u64* out, u64* scratch) {
  const int t = threadIdx.x;
  u64 lo = 0, hi = 0;
  if (t < 64) {
    // lo = p_t = sum_{i<=t} a_i b_{t-i};  hi = p_{64+t} = sum_{i>t} a_i b_{64+t-i}
    for (int i = 0; i <= t; ++i) lo += a[i] * b[t - i];
    for (int i = t + 1; i < 64; ++i) hi += a[i] * b[64 + t - i];
  }
  __syncthreads();
  if (t < 64) { scratch[t] = lo; scratch[64 + t] = (t < 63) ? hi : 0; }
  __syncthreads();
  if (t < 64) {
    const u64* h = scratch + 64;
    u64 v = scratch[t] - gr_hg(h, t);
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
    lo = v;
  }
  __syncthreads();
  if (t < 64) out[t] = lo;
  __syncthreads();
}

// Multiplication matrix of a constant a: M[b][c] = coefficient c of a * x^b (block-cooperative,
// 64 threads).  Row b+1 = x * row b: shift up one coefficient, the top coefficient u wraps as
// x^64 = -(1 + x + x^3 + x^4).
__device__ inline void gr_mulmat_block(const u64* a, u64* M /*64x64 row-major*/) {
  const int t = threadIdx.x;
  if (t < 64) M[t] = a[t];
  __syncthreads();
  for (int b = 1; b < 64; ++b) {
    u64 v = 0;
    if (t < 64) {
      const u64* prev = M + (b - 1) * 64;
      const u64 u = prev[63];
      v = (t > 0) ? prev[t - 1] : 0;
      if (t == 0 || t == 1 || t == 3 || t == 4) v -= u;
    }
    __syncthreads();
    if (t < 64) M[b * 64 + t] = v;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// SHA-256 (FIPS 180-4)
// ---------------------------------------------------------------------------------------------
__device__ __constant__ static const u32 SHA_K[64] = {
    0x428a2f98u, 0x71374491u, 0xb5c0fbcfu, 0xe9b5dba5u, 0x3956c25bu, 0x59f111f1u, 0x923f82a4u,
    0xab1c5ed5u, 0xd807aa98u, 0x12835b01u, 0x243185beu, 0x550c7dc3u, 0x72be5d74u, 0x80deb1feu,
    0x9bdc06a7u, 0xc19bf174u, 0xe49b69c1u, 0xefbe4786u, 0x0fc19dc6u, 0x240ca1ccu, 0x2de92c6fu,
    0x4a7484aau, 0x5cb0a9dcu, 0x76f988dau, 0x983e5152u, 0xa831c66du, 0xb00327c8u, 0xbf597fc7u,
    0xc6e00bf3u, 0xd5a79147u, 0x06ca6351u, 0x14292967u, 0x27b70a85u, 0x2e1b2138u, 0x4d2c6dfcu,
    0x53380d13u, 0x650a7354u, 0x766a0abbu, 0x81c2c92eu, 0x92722c85u, 0xa2bfe8a1u, 0xa81a664bu,
    0xc24b8b70u, 0xc76c51a3u, 0xd192e819u, 0xd6990624u, 0xf40e3585u, 0x106aa070u, 0x19a4c116u,
    0x1e376c08u, 0x2748774cu, 0x34b0bcb5u, 0x391c0cb3u, 0x4ed8aa4au, 0x5b9cca4fu, 0x682e6ff3u,
    0x748f82eeu, 0x78a5636fu, 0x84c87814u, 0x8cc70208u, 0x90befffau, 0xa4506cebu, 0xbef9a3f7u,
    0xc67178f2u};

__device__ __forceinline__ u32 rotr32(u32 x, int n) { return __funnelshift_r(x, x, n); }

__device__ inline void sha256_init(u32 h[8]) {
  h[0] = 0x6a09e667u; h[1] = 0xbb67ae85u; h[2] = 0x3c6ef372u; h[3] = 0xa54ff53au;
  h[4] = 0x510e527fu; h[5] = 0x9b05688cu; h[6] = 0x1f83d9abu; h[7] = 0x5be0cd19u;
}

// Compress one 64-byte block given as 16 big-endian words.
__device__ inline void sha256_compress(u32 h[8], const u32 wblk[16]) {
  u32 w[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) w[i] = wblk[i];
  u32 a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
#pragma unroll
  for (int t = 0; t < 64; ++t) {
    u32 wt;
    if (t < 16) {
      wt = w[t];
    } else {
      const u32 w15 = w[(t - 15) & 15], w2 = w[(t - 2) & 15];
      const u32 s0 = rotr32(w15, 7) ^ rotr32(w15, 18) ^ (w15 >> 3);
      const u32 s1 = rotr32(w2, 17) ^ rotr32(w2, 19) ^ (w2 >> 10);
      wt = w[t & 15] + s0 + w[(t - 7) & 15] + s1;
      w[t & 15] = wt;
    }
    const u32 S1 = rotr32(e, 6) ^ rotr32(e, 11) ^ rotr32(e, 25);
    const u32 ch = (e & f) ^ (~e & g);
    const u32 t1 = hh + S1 + ch + SHA_K[t] + wt;
    const u32 S0 = rotr32(a, 2) ^ rotr32(a, 13) ^ rotr32(a, 22);
    const u32 mj = (a & b) ^ (a & c) ^ (b & c);
    const u32 t2 = S0 + mj;
    hh = g; g = f; f = e; e = d + t1; d = c; c = b; b = a; a = t1 + t2;
  }
  h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
}

__device__ __forceinline__ u32 bswap32(u32 x) { return __byte_perm(x, 0, 0x0123); }

}  // namespace mpc3
