// H of Pi_Rec (Sec. 2, verifiable reconstruction): SHA-256 (FIPS 180-4) of each 1024-byte leaf
// of the little-endian byte image of a u64 array, then a binary tree whose node is
// SHA-256(left || right), an odd node being promoted unchanged.  One thread hashes one leaf and
// each CTA reduces its 64 aligned leaves to their subtree root (the tree's six lowest levels;
// for the ragged last CTA the promotion rule applies inside it, as it would globally); one CTA
// builds the rest of the tree.  Digests are kept as 8 big-endian 32-bit words.
#include "kernels.h"

namespace mpc3 {

namespace {

constexpr long long LEAF_BYTES = HASH_LEAF_BYTES;
constexpr long long LEAF_WORDS = LEAF_BYTES / 8;
constexpr int HB = (int)HASH_CTA_LEAVES;   // leaves (threads) per CTA of k_hash_leaves

// h = SHA-256(l || r) of two digests (one data block and one padding block)
__device__ __forceinline__ void node_hash(const u32* l, const u32* r, u32 h[8]) {
  sha256_init(h);
  u32 blk[16];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    blk[q] = l[q];
    blk[8 + q] = r[q];
  }
  sha256_compress(h, blk);
#pragma unroll
  for (int q = 0; q < 16; ++q) blk[q] = 0;
  blk[0] = 0x80000000u;
  blk[15] = 512u;
  sha256_compress(h, blk);
}

__global__ void __launch_bounds__(HB)
k_hash_leaves(const u64* __restrict__ data, long long n, long long nleaves,
              u32* __restrict__ out) {
  __shared__ u32 dg[HB][8];
  const long long leaf = blockIdx.x * (long long)HB + threadIdx.x;
  if (leaf < nleaves) {
    const long long w0 = leaf * LEAF_WORDS;
    long long nw = n - w0;
    if (nw > LEAF_WORDS) nw = LEAF_WORDS;
    if (nw < 0) nw = 0;
    u32 h[8];
    sha256_init(h);
    u32 blk[16];
    long long i = 0;
    // full 64-byte blocks; the next block's words are loaded before this one is compressed
    u64 nx[8];
    if (nw >= 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q) nx[q] = data[w0 + q];
    }
    for (; i + 8 <= nw; i += 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        blk[2 * q] = bswap32((u32)nx[q]);
        blk[2 * q + 1] = bswap32((u32)(nx[q] >> 32));
      }
      if (i + 16 <= nw) {
#pragma unroll
        for (int q = 0; q < 8; ++q) nx[q] = data[w0 + i + 8 + q];
      }
      sha256_compress(h, blk);
    }
    // tail: r = nw - i words (0..7), then 0x80, zeros, 64-bit length
    const int r = (int)(nw - i);
#pragma unroll
    for (int q = 0; q < 16; ++q) blk[q] = 0;
    for (int q = 0; q < r; ++q) {
      const u64 v = data[w0 + i + q];
      blk[2 * q] = bswap32((u32)v);
      blk[2 * q + 1] = bswap32((u32)(v >> 32));
    }
    blk[2 * r] = 0x80000000u;
    const u64 bits = (u64)nw * 64ull;
    if (2 * r + 1 > 14) {           // length does not fit: extra block
      sha256_compress(h, blk);
#pragma unroll
      for (int q = 0; q < 16; ++q) blk[q] = 0;
    }
    blk[14] = (u32)(bits >> 32);
    blk[15] = (u32)bits;
    sha256_compress(h, blk);
#pragma unroll
    for (int q = 0; q < 8; ++q) dg[threadIdx.x][q] = h[q];
  }
  __syncthreads();
  // the six lowest tree levels over this CTA's leaves
  long long rem = nleaves - blockIdx.x * (long long)HB;
  int cnt = rem < HB ? (int)rem : HB;
  while (cnt > 1) {
    const int half = cnt / 2;
    const int p = threadIdx.x;
    u32 h[8];
    if (p < half) node_hash(dg[2 * p], dg[2 * p + 1], h);
    u32 carry[8];
    if ((cnt & 1) && p == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) carry[q] = dg[cnt - 1][q];
    }
    __syncthreads();
    if (p < half) {
#pragma unroll
      for (int q = 0; q < 8; ++q) dg[p][q] = h[q];
    }
    if ((cnt & 1) && p == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) dg[half][q] = carry[q];
    }
    __syncthreads();
    cnt = half + (cnt & 1);
  }
  if (threadIdx.x < 8) out[blockIdx.x * 8 + threadIdx.x] = dg[0][threadIdx.x];
}

// One CTA: levels of the Merkle tree over `cnt` digests in buf (ping-pong with buf2).
__global__ void k_hash_tree(u32* buf, u32* buf2, long long cnt, u32* digest) {
  u32* cur = buf;
  u32* nxt = buf2;
  while (cnt > 1) {
    const long long half = cnt / 2;
    for (long long p = threadIdx.x; p < half; p += blockDim.x) {
      u32 h[8];
      node_hash(cur + (2 * p) * 8, cur + (2 * p + 1) * 8, h);
#pragma unroll
      for (int q = 0; q < 8; ++q) nxt[p * 8 + q] = h[q];
    }
    if ((cnt & 1) && threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) nxt[half * 8 + q] = cur[(cnt - 1) * 8 + q];
    }
    __syncthreads();
    cnt = half + (cnt & 1);
    u32* t = cur;
    cur = nxt;
    nxt = t;
    __syncthreads();
  }
  if (threadIdx.x < 8) digest[threadIdx.x] = cur[threadIdx.x];
}

// Compare three (received value's hash, received hash) pairs; any mismatch sets `flag`.
__global__ void k_digest_check(const u32* a0, const u32* b0, const u32* a1, const u32* b1,
                               const u32* a2, const u32* b2, u32* status, u32 flag) {
  const int t = threadIdx.x;
  bool bad = false;
  if (t < 8) bad = (a0[t] != b0[t]) || (a1[t] != b1[t]) || (a2[t] != b2[t]);
  if (bad) atomicOr(status, flag);
}

}  // namespace

size_t hash_scratch_words(long long n) { return (size_t)hash_scratch_words_for(n); }

void launch_hash_u64(cudaStream_t st, const u64* data, long long n, u32* scratch, u32* digest) {
  long long leaves = (8 * n + LEAF_BYTES - 1) / LEAF_BYTES;
  if (leaves < 1) leaves = 1;
  const long long nb = (leaves + HB - 1) / HB;   // subtree roots, one per CTA
  k_hash_leaves<<<(unsigned)nb, HB, 0, st>>>(data, n, leaves, scratch);
  k_hash_tree<<<1, 256, 0, st>>>(scratch, scratch + 8 * nb, nb, digest);
}

void launch_digest_check(cudaStream_t st, const u32* a0, const u32* b0, const u32* a1,
                         const u32* b1, const u32* a2, const u32* b2, u32* status, u32 flag) {
  k_digest_check<<<1, 32, 0, st>>>(a0, b0, a1, b1, a2, b2, status, flag);
}

}  // namespace mpc3
