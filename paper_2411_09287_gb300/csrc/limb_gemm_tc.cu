// Exact Z_2^64 GEMM on the 5th-generation tensor cores (tcgen05, kind::f16 with f16 inputs,
// f32 accumulators in tensor memory): the "limb tensor-core path" of the local products of
// Pi_Inner (Fig. DPP, Sec. 4.1).
//
// Each u64 operand value is split into 8 balanced signed digits d_0..d_7 in [-128, 127] with
// v = sum_i 2^(8i) d_i mod 2^64 (carry-propagating split; the carry out of d_7 vanishes mod 2^64).
// f16 holds every such digit exactly.  Only digit pairs with i + j < 8 contribute mod 2^64:
//   C = sum_{s<8} 2^(8s) C_s,   C_s = sum_{i+j=s} A_i B_j      (36 digit-plane products).
// Each C_s has its own TMEM accumulator (8 x 64 columns = all 512).  An accumulation runs over
// at most 64 of K (two chunks of 32), so |C_s| <= (s + 1) * 64 * 2^14: every f32 partial sum is
// an exact integer.  For s <= 3 (|C_s| <= 2^22), adding 1.5 * 2^23 turns it into an
// integer-valued float whose bit pattern minus 0x4B400000 is that integer; for s >= 4
// (|C_s| <= 2^23) a float-to-int conversion does it.  After each accumulation the accumulators
// are drained into 64-bit registers, which wrap mod 2^64 as required:
//   acc += (v0 + 2^8 v1) + 2^16 (v2 + 2^8 v3) + 2^32 (v4 + 2^8 v5) + 2^48 (v6 + 2^8 v7),
// each bracket computed in 32-bit arithmetic (|v0 + 2^8 v1|, |v2 + 2^8 v3| < 2^31; the two high
// brackets only matter mod 2^32 and 2^16).
//
// CTA = one 128 x 64 output tile, 10 warps with fixed roles:
//   warps 0..7  drain: warp w reads TMEM lanes 32 (w % 4) .. +31 (= tile rows) and columns
//               32 (w / 4) .. +31 of every accumulator;
//   warp 8      TMA producer: 8 + 8 digit-plane tiles per K chunk into a 2-stage ring (64-byte
//               swizzle, 96 KB per stage);
//   warp 9      MMA issuer (one thread): accumulator group GA = {0, 1, 6, 7} then GB = {2, 3, 4, 5}
//               (18 digit pairs each), each committed to its own mbarrier, so that the drain of
//               one group overlaps the MMAs of the other.
// Every mbarrier wait is bounded (clock64, about one second) and also gives up once another
// warp has recorded a failure; a failure sets err_flag in *err, the CTA lets its TMA copies and
// MMAs finish (bounded), frees its tensor memory and returns without writing its tile.
#include <climits>
#include <type_traits>

#include <cstring>

#include "kernels.h"
#include "tcgen05.cuh"

namespace mpc3 {

namespace {

using namespace tc;

constexpr int TC_BM = 128, TC_BN = 64, TC_BK = 32;
constexpr int A_TILE = TC_BM * TC_BK * 2;   // 8 KB per digit plane
constexpr int B_TILE = TC_BN * TC_BK * 2;   // 4 KB per digit plane
constexpr int STAGE = 8 * (A_TILE + B_TILE);   // 96 KB
constexpr int NSTAGE = 2;
constexpr int NDRAIN = 8;
constexpr int TC_THREADS = (NDRAIN + 2) * 32;

// Instruction descriptor, kind::f16: f32 accumulator, f16 A and B, both K-major, M = 128, N = 64.
constexpr unsigned IDESC = (1u << 4) | ((unsigned)(TC_BN >> 3) << 17) |
                           ((unsigned)(TC_BM >> 4) << 24);

// D (+)= A B; acc = 0 overwrites the accumulator, 1 adds to it
__device__ __forceinline__ void mma_f16(unsigned d_tmem, u64 adesc, u64 bdesc, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc));
}
// Bit pattern of (v + 1.5 * 2^23) for an integer-valued f32 v in [-2^22, 2^22]: equals
// v + MAGIC_I exactly (the sum lies in [2^23, 2^24], where every integer is a float).
constexpr unsigned MAGIC_I = 0x4B400000u;
constexpr unsigned PAIR_BIAS = MAGIC_I + 256u * MAGIC_I;   // bias of v_s + 2^8 v_(s+1), mod 2^32
__device__ __forceinline__ int f2i_biased(unsigned bits) {
  return __float_as_int(__uint_as_float(bits) + 12582912.0f);
}
// the integer value of an integer-valued f32 (exact for |v| <= 2^24)
__device__ __forceinline__ unsigned f32_int(unsigned bits) {
  int r;
  asm("cvt.rni.s32.f32 %0, %1;\n" : "=r"(r) : "f"(__uint_as_float(bits)));
  return (unsigned)r;
}

// TMEM column of accumulator s: group GA = {0, 1, 6, 7} in columns 0..255, GB = {2..5} above
__host__ __device__ constexpr int acc_col(int s) {
  return s == 0 ? 0 : s == 1 ? 64 : s == 6 ? 128 : s == 7 ? 192 : 256 + (s - 2) * 64;
}
// digit weight of the g-th accumulator of group G (GA = {0, 1, 6, 7}, GB = {2, 3, 4, 5})
__host__ __device__ constexpr int group_s(int G, int g) { return G == 0 ? (g < 2 ? g : g + 4) : g + 2; }

// Drain of accumulator group G for the 16 TMEM columns at tl + col: acc[j] += G = 0:
// (v0 + 2^8 v1) + 2^48 (v6 + 2^8 v7), G = 1: 2^16 (v2 + 2^8 v3) + 2^32 (v4 + 2^8 v5).
template <int G>
__device__ __forceinline__ void drain16(unsigned tl, int col, u64* acc) {
  constexpr int s0 = G == 0 ? 0 : 2, s1 = G == 0 ? 6 : 4;
#pragma unroll
  for (int h8 = 0; h8 < 16; h8 += 8) {   // 8 columns at a time (bounded register use)
    unsigned x0[8], x1[8], y0[8], y1[8];
    tmem_ld8(tl + (unsigned)(acc_col(s0) + col + h8), x0);
    tmem_ld8(tl + (unsigned)(acc_col(s0 + 1) + col + h8), x1);
    tmem_ld8(tl + (unsigned)(acc_col(s1) + col + h8), y0);
    tmem_ld8(tl + (unsigned)(acc_col(s1 + 1) + col + h8), y1);
    tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      // + ws (G = 0) or 2^16 ws (G = 1), ws sign-extended; + 2^48 whi (G = 0) or 2^32 whi (G = 1)
      const unsigned ws =
          (unsigned)f2i_biased(x0[j]) + (unsigned)f2i_biased(x1[j]) * 256u - PAIR_BIAS;
      const unsigned whi = f32_int(y0[j]) + f32_int(y1[j]) * 256u;
      acc[h8 + j] += (G == 0 ? (u64)(long long)(int)ws : (u64)(long long)(int)ws << 16) +
                     ((u64)(G == 0 ? (whi << 16) : whi) << 32);
    }
  }
}

// The same for the merged pairs of a bit-operand product: accumulator s (s even) holds
// C_s + 2^8 C_(s+1) (|.| < 2^22, the magic-number pattern suffices).
template <int G>
__device__ __forceinline__ void drain16_pairs(unsigned tl, int col, u64* acc) {
  constexpr int s0 = G == 0 ? 0 : 2, s1 = G == 0 ? 6 : 4;
#pragma unroll
  for (int h8 = 0; h8 < 16; h8 += 8) {
    unsigned x0[8], y0[8];
    tmem_ld8(tl + (unsigned)(acc_col(s0) + col + h8), x0);
    tmem_ld8(tl + (unsigned)(acc_col(s1) + col + h8), y0);
    tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const unsigned ws = (unsigned)f2i_biased(x0[j]) - MAGIC_I;
      const unsigned whi = (unsigned)f2i_biased(y0[j]) - MAGIC_I;
      acc[h8 + j] += (G == 0 ? (u64)(long long)(int)ws : (u64)(long long)(int)ws << 16) +
                     ((u64)(G == 0 ? (whi << 16) : whi) << 32);
    }
  }
}

// All MMAs of one accumulator group for one K chunk, fully unrolled: a_desc / b_desc are the
// descriptors of digit plane 0 of the stage; plane i is A_TILE (B_TILE) bytes further on, and
// each k16 step advances 32 bytes inside the swizzled rows.
// With A0 set, A has digit plane 0 only (0/1 entries) and the odd B planes hold 256 B_s: the pair
// (s, s + 1), s even, goes into the accumulator of s as C_s + 2^8 C_(s+1) (|.| <= 64 (128 +
// 2^15) < 2^22 per 64 of K), four accumulators instead of eight.
// fresh = 0 adds the chunk to what the accumulators hold instead of starting them anew.
// KK >= 0 issues only the MMAs of that k16 step (K words 16 KK .. 16 KK + 15 of the chunk).
template <int G, bool A0 = false, int KK = -1>
__device__ __forceinline__ void issue_group(unsigned tmem, u64 a_desc, u64 b_desc,
                                            unsigned fresh = 1) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int s = group_s(G, g);
    const int sa = A0 ? (s & ~1) : s;   // target accumulator
#pragma unroll
    for (int kk = (KK < 0 ? 0 : KK); kk < (KK < 0 ? TC_BK / 16 : KK + 1); ++kk) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (i <= s && (!A0 || i == 0)) {
          const u64 ad = a_desc + (u64)((i * A_TILE) >> 4) + (u64)(kk * 2);
          const u64 bd = b_desc + (u64)(((s - i) * B_TILE) >> 4) + (u64)(kk * 2);
          const bool first = kk == 0 && i == 0 && sa == s;
          mma_f16(tmem + (unsigned)acc_col(sa), ad, bd, first ? (fresh ^ 1u) : 1u);
        }
      }
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
k_limb_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               long long M, long long N, long long Kp, u64* __restrict__ C, long long ldc,
               unsigned* __restrict__ err, unsigned err_flag) {
  // split K over gridDim.z: this CTA takes chunks [cbeg, cbeg + nchunks); with more than one
  // split the partial tiles are added atomically into C (zeroed by the host)
  extern __shared__ unsigned char dsm[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) u64 full_bar[NSTAGE], empty_bar[NSTAGE];
  __shared__ __align__(8) u64 accf_bar[2], acce_bar[2], done_bar;
  __shared__ unsigned tmem_slot;
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const long long m0 = (long long)blockIdx.x * TC_BM;
  const long long n0 = (long long)blockIdx.y * TC_BN;
  const int nall = (int)(Kp / TC_BK);
  const int cbeg = (int)((long long)nall * blockIdx.z / gridDim.z);
  const int nchunks = (int)((long long)nall * (blockIdx.z + 1) / gridDim.z) - cbeg;
  const bool split = gridDim.z > 1;

  if (tid == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    for (int g = 0; g < 2; ++g) {
      mbar_init(&accf_bar[g], 1);
      mbar_init(&acce_bar[g], NDRAIN);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(
        smem_u32(&tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = tmem_slot;

  auto fail = [&]() {
    *abort = 1;
    atomicOr(err, err_flag);
  };

  if (warp == NDRAIN) {
    // ---- TMA producer ----
    if (lane == 0) {
      int last = -1;
      for (int c = 0; c < nchunks; ++c) {
        const int st = c % NSTAGE;
        if (c >= NSTAGE && !mbar_wait(&empty_bar[st], (unsigned)(((c / NSTAGE) + 1) & 1), abort)) {
          fail();
          break;
        }
        unsigned char* As = base + st * STAGE;
        unsigned char* Bs = As + 8 * A_TILE;
        mbar_expect_tx(&full_bar[st], (unsigned)STAGE);
        const int kx = (cbeg + c) * TC_BK;
#pragma unroll 1
        for (int i = 0; i < 8; ++i) {
          tma_load_3d(As + i * A_TILE, &tmA, &full_bar[st], kx, (int)m0, i);
          tma_load_3d(Bs + i * B_TILE, &tmB, &full_bar[st], kx, (int)n0, i);
        }
        last = c;
      }
      // the copies of the last chunk issued into each stage must land before the CTA exits
      for (int c = last; c >= 0 && c > last - NSTAGE; --c)
        mbar_wait_plain(&full_bar[c % NSTAGE], (unsigned)((c / NSTAGE) & 1));
    }
  } else if (warp == NDRAIN + 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const u64 d0 = smem_desc(base, 64);
      for (int c = 0; c < nchunks; ++c) {
        const int st = c % NSTAGE;
        if (!mbar_wait(&full_bar[st], (unsigned)((c / NSTAGE) & 1), abort)) { fail(); break; }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const u64 ad = d0 + (u64)((st * STAGE) >> 4);
        const u64 bd = ad + (u64)((8 * A_TILE) >> 4);
        // accumulation v takes chunks 2v and 2v + 1 (K <= 64 per accumulation)
        const bool first = !(c & 1), last = (c & 1) || c == nchunks - 1;
        const int v = c >> 1;
        if (first && v > 0 && !mbar_wait(&acce_bar[0], (unsigned)((v - 1) & 1), abort)) { fail(); break; }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        issue_group<0>(tmem, ad, bd, first ? 1u : 0u);
        if (last) mma_commit(&accf_bar[0]);
        if (first && v > 0 && !mbar_wait(&acce_bar[1], (unsigned)((v - 1) & 1), abort)) { fail(); break; }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        issue_group<1>(tmem, ad, bd, first ? 1u : 0u);
        if (last) mma_commit(&accf_bar[1]);
        mma_commit(&empty_bar[st]);   // the stage is free once these MMAs have read it
      }
      // every MMA issued must complete before the tensor memory is released
      mma_commit(&done_bar);
      mbar_wait_plain(&done_bar, 0u);
    }
  } else {
    // ---- drain warps ----
    const int q = warp & 3, h = warp >> 2;
    const unsigned tl = tmem + ((unsigned)(q * 32) << 16) + (unsigned)(h * 32);
    u64 acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = 0;
    bool ok = true;
    const int nacc = (nchunks + 1) / 2;
    for (int v = 0; v < nacc && ok; ++v) {
      const unsigned par = (unsigned)(v & 1);
#pragma unroll 1
      for (int g = 0; g < 2; ++g) {
        ok = __all_sync(0xffffffffu, mbar_wait(&accf_bar[g], par, abort));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
        for (int c16 = 0; c16 < 2; ++c16) {
          if (g == 0) drain16<0>(tl, c16 * 16, acc + c16 * 16);
          else drain16<1>(tl, c16 * 16, acc + c16 * 16);
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce_bar[g]);
      }
    }
    if (ok && !*abort) {
      // through a per-warp 32-row x 4-column block of shared memory, so that every store (or
      // atomic) instruction covers 16 rows x 32 contiguous bytes
      const long long r = m0 + q * 32 + lane;
      const long long cb = n0 + h * 32;
      unsigned char* os = base + NSTAGE * STAGE + warp * (32 * 48);
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 4) {
#pragma unroll
        for (int qq = 0; qq < 2; ++qq)
          *reinterpret_cast<ulonglong2*>(os + lane * 48 + qq * 16) =
              make_ulonglong2(acc[c0 + 2 * qq], acc[c0 + 2 * qq + 1]);
        __syncwarp();
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
          const int rr = pass * 16 + (lane >> 1), ch = lane & 1;
          const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(os + rr * 48 + ch * 16);
          const long long row = m0 + q * 32 + rr, col = cb + c0 + 2 * ch;
          if (row < M) {
            u64* dst = C + row * ldc + col;
            if (split) {
              if (col < N) atomicAdd(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)w.x);
              if (col + 1 < N) atomicAdd(reinterpret_cast<unsigned long long*>(dst + 1), (unsigned long long)w.y);
            } else {
              if (col < N) dst[0] = w.x;
              if (col + 1 < N) dst[1] = w.y;
            }
          }
        }
        __syncwarp();
      }
      (void)r;
    } else if (!ok) {
      if (lane == 0) fail();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
}

// ---- digit split ------------------------------------------------------------------------------
__device__ __forceinline__ u64 load_opnd(const Opnd& o, long long r, long long c, long long R,
                                         long long Cn) {
  if (r >= R || c >= Cn) return 0;
  const long long off = o.trans ? (c * o.ld + r) : (r * o.ld + c);
  u64 v = o.p0[off];
  if (o.p1) {
    const u64 w = o.p1[off];
    v = (o.s1 == 1ull) ? v + w : ((o.s1 == ~0ull) ? v - w : v + o.s1 * w);
  }
  if (o.scale != 1ull) v = (o.scale == ~0ull) ? (0ull - v) : o.scale * v;
  return v;
}

// 8 consecutive u64 values -> 8 digit planes of 8 f16 each (one 16-byte unit per plane).
// The balanced digits of v are the bytes of v + 0x8080808080808080 minus 128 (the digit set
// [-128, 127] is a complete residue system, so this is the carry-propagating split).  A byte b
// placed under the f16 exponent byte 0x64 is the f16 of 1024 + b (the spacing of f16 values on
// [1024, 2048) is 1), so one packed f16 subtraction of 1152 per pair of digits leaves b - 128
// exactly.  Per pair of words and 32-bit half: four byte permutes place bytes (0, 2) and (1, 3)
// of each word under the exponent byte, four more pair the two words along K, four subtractions.
__device__ __forceinline__ unsigned f16x2_minus_1152(unsigned x) {
  unsigned r;
  asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(r) : "r"(x), "r"(0x64806480u));
  return r;
}
__device__ __forceinline__ unsigned f16x2_times_256(unsigned x) {   // exact for |x| <= 128
  unsigned r;
  asm("mul.rn.f16x2 %0, %1, %2;\n" : "=r"(r) : "r"(x), "r"(0x5C005C00u));
  return r;
}
// scale_odd: the odd digit planes are stored times 2^8 (B of a bit-operand product)
__device__ __forceinline__ void split8_store(const u64 v[8], unsigned char* plane0,
                                             long long plane_stride, int off,
                                             bool scale_odd = false) {
  unsigned pk[8][4];   // [plane][k pair m]: f16 digits of words 2m (low half) and 2m + 1
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const u64 a = v[2 * m] + 0x8080808080808080ull, b = v[2 * m + 1] + 0x8080808080808080ull;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned xa = (unsigned)(a >> (32 * h)), xb = (unsigned)(b >> (32 * h));
      const unsigned a02 = __byte_perm(xa, 0x64u, 0x4240), a13 = __byte_perm(xa, 0x64u, 0x4341);
      const unsigned b02 = __byte_perm(xb, 0x64u, 0x4240), b13 = __byte_perm(xb, 0x64u, 0x4341);
      pk[4 * h + 0][m] = f16x2_minus_1152(__byte_perm(a02, b02, 0x5410));
      pk[4 * h + 2][m] = f16x2_minus_1152(__byte_perm(a02, b02, 0x7632));
      pk[4 * h + 1][m] = f16x2_minus_1152(__byte_perm(a13, b13, 0x5410));
      pk[4 * h + 3][m] = f16x2_minus_1152(__byte_perm(a13, b13, 0x7632));
    }
  }
  if (scale_odd) {
#pragma unroll
    for (int i = 1; i < 8; i += 2)
#pragma unroll
      for (int m = 0; m < 4; ++m) pk[i][m] = f16x2_times_256(pk[i][m]);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
    *reinterpret_cast<uint4*>(plane0 + i * plane_stride + off) =
        make_uint4(pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
}
// 8 bits (k = 0..7, bit k of `bits`) -> the 16-byte unit of digit plane 0 (f16 0 or 1); the
// other planes of such an operand are zero.
__device__ __forceinline__ uint4 bits_plane0(unsigned bits) {
  unsigned pk[4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
    pk[m] = ((bits >> (2 * m)) & 1u) * 0x3C00u + ((bits >> (2 * m + 1)) & 1u) * 0x3C000000u;
  return make_uint4(pk[0], pk[1], pk[2], pk[3]);
}

// planes[i][row][k'] (f16), row-major with pitch Kp; element (row, k') of the concatenated
// operand: term t = k' / K, column k' mod K; values beyond nterms*K are zero.
__global__ void k_split_digits(GemmTerm t0, GemmTerm t1, int nterms, int which /*0 A, 1 B*/,
                               long long R, long long K, long long Kp,
                               unsigned short* __restrict__ planes) {
  const long long chunks = Kp / 8;
  const long long total = R * chunks;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
       w += (long long)gridDim.x * blockDim.x) {
    // consecutive threads take consecutive rows for B (coalesced column reads of a row-major
    // K x N operand) and consecutive k chunks for A
    long long row, kc;
    if (which) { row = w % R; kc = w / R; } else { row = w / chunks; kc = w % chunks; }
    u64 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const long long kk = kc * 8 + q;
      v[q] = 0;
      if (kk < (long long)nterms * K) {
        const GemmTerm& T = (kk < K) ? t0 : t1;
        const long long k = kk < K ? kk : kk - K;
        v[q] = which ? load_opnd(T.B, k, row, K, R) : load_opnd(T.A, row, k, R, K);
      }
    }
    split8_store(v, reinterpret_cast<unsigned char*>(planes + row * Kp + kc * 8), R * Kp * 2, 0);
  }
}

// The B split for a row-major K x R source (trans = 0): a 64 k x 32 r block goes through shared
// memory, so that the reads run along r and every plane row gets 128 contiguous bytes per 8
// threads (the direct split writes one 16-byte unit per row and thread).
__global__ void __launch_bounds__(256)
k_split_digits_bt(GemmTerm t0, GemmTerm t1, int nterms, long long R, long long K, long long Kp,
                  unsigned short* __restrict__ planes) {
  __shared__ u64 tile[32][65];
  const long long r0 = (long long)blockIdx.x * 32;
  const long long k0 = (long long)blockIdx.y * 64;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int kl = w * 8 + j;
    const long long kk = k0 + kl;
    u64 v = 0;
    if (kk < (long long)nterms * K && r0 + lane < R) {
      const GemmTerm& T = (kk < K) ? t0 : t1;
      v = load_opnd(T.B, kk < K ? kk : kk - K, r0 + lane, K, R);
    }
    tile[lane][kl] = v;
  }
  __syncthreads();
  const int rl = threadIdx.x >> 3, kc = threadIdx.x & 7;
  const long long r = r0 + rl, kk0 = k0 + kc * 8;
  if (r < R && kk0 < Kp) {
    u64 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = tile[rl][kc * 8 + q];
    split8_store(v, reinterpret_cast<unsigned char*>(planes + r * Kp + kk0), R * Kp * 2, 0);
  }
}

// out[i] = acc_sign*out[i] + add0 + add1 + prf_sign*PRF(i) (the protocol epilogue of gemm_u64).
__global__ void k_apply_epilogue(long long M, long long N, Epi epi) {
  const long long total = M * N;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < (total + 7) / 8;
       w += (long long)gridDim.x * blockDim.x) {
    const long long i0 = w * 8;
    u64 pr[8];
    bool block = epi.prf_sign && (N % 8 == 0) && (epi.ldc == N);
    if (block) prf_block8(epi.key, epi.tag, epi.obj, (u64)(i0 >> 3), pr);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const long long i = i0 + q;
      if (i >= total) break;
      const long long r = i / N, c = i % N;
      const long long idx = r * epi.ldc + c;
      u64 v = epi.out[idx];
      v = (epi.acc_sign == 1ull) ? v : ((epi.acc_sign == ~0ull) ? 0ull - v : epi.acc_sign * v);
      if (epi.add0) v += epi.add0[epi.ld_add0 ? r * epi.ld_add0 + c : idx];
      if (epi.add1) v += epi.add1[idx];
      if (epi.prf_sign) {
        const u64 p = block ? pr[q] : prf_word(epi.key, epi.tag, epi.obj, (u64)idx);
        v += epi.prf_sign * p;
      }
      epi.out[idx] = v;
    }
  }
}

bool make_map(CUtensorMap* map, void* planes, long long rows, long long Kp, int box_rows) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, 8};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(rows * Kp * 2)};
  cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};   // 64-byte rows
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, planes, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---- GR-matrix products out = add0 + A . M with K = N = 64 (folds, powers tables) -------------
// out[i][c] = add0[i][c] + sum_k A[i][k] M[k][c] for rows i < R, with A[i][k] = p0[i][k] + s1 p1[i][k]
// (row stride lda) and M a 64 x 64 u64 matrix (the multiplication matrix of a GR element).
// Same digit scheme and accumulator groups as k_limb_gemm_tc; the differences:
//   - persistent CTAs loop over 128-row tiles; K = 64 is two chunks of 32;
//   - B = M^T is split into digit planes in shared memory (64 KB) when a CTA's tile range enters
//     a new matrix group (rows rho of group rho / mrows use matrix rho / mrows; one group by
//     default), after the MMAs of the previous tile have finished reading the old planes;
//   - rows go through row maps: A row rho is read at p0 + map_in(rho) and its result written at
//     out + map_out(rho) (map(rho) = (rho % q) s1 + (rho / q) s2 words), which lets one launch
//     gather strided rows or scatter a transposed order;
//   - three producer warps load the A rows from global memory (all of a chunk's loads issued
//     before the first is used) and split them into the swizzled digit planes directly (no
//     digit-plane copy in HBM); the MMA issuer is as before; eight drain warps (each 32 rows x 32
//     columns) add add0 and store the tile;
//   - a_bits mode (A = the bits of one word per row): A has digit plane 0 only, so the producers
//     write that plane alone and the issuer runs the 8 pairs (0, s) instead of 36, merged two by
//     two into four accumulators (odd B planes stored times 2^8), which halves the drain.  Its
//     tiles can leave by TMA tensor stores: the drain warps write the tile into four 128-byte
//     swizzled boxes (16 words x 128 rows) in the A stages' unused planes, and one thread stores
//     them while the next tile is drained.
constexpr int GM_NDRAIN = 8;                              // drain warps: 32 rows x GM_DC columns
constexpr int GM_DC = 256 / GM_NDRAIN;                    // columns per drain warp (32)
constexpr int GM_PROD = 3;                                // producer warps
constexpr int GM_THREADS = (GM_NDRAIN + GM_PROD + 1) * 32;   // 384
constexpr int GM_BCHUNK = 8 * B_TILE;                     // 32 KB: B planes of one K chunk
// per drain warp: a 32-row x 4-column u64 block for the transposed (coalesced) stores, rows 48
// bytes apart so that both the row-wise writes and the 16-byte-chunk reads are conflict-free
constexpr int GM_OROW = 48;
constexpr int GM_OSTAGE = 32 * GM_OROW;

// byte offset of 16-byte unit u (8 f16 along K) of row r inside a K-major 64-byte-swizzled tile
__device__ __forceinline__ int sw64_off(int r, int u) {
  return (r >> 3) * 512 + (r & 7) * 64 + ((u ^ ((r >> 1) & 3)) << 4);
}

__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ long long rowmap(const GrRowMap& m, long long rho) {
  return m.q ? (rho % m.q) * m.s1 + (rho / m.q) * m.s2 : rho * m.s1;
}

// MODE 0: plain product, 1: fold (p0 - p1), 2: bit operand.  One instantiation per mode keeps
// each kernel's code (and instruction-cache footprint) to the paths it runs.
// TMA (MODE 0 and 1): one A stage, handled by K halves; the other stage's 64 KB holds slots of
// raw A rows, one half-unit (16 words x 128 rows of p0, and of p1 in a fold) per slot, loaded by
// TMA from the row-mapped input (tensor maps tm0 for p0, tm1 for p1: boxes of 16 words x 128 rows,
// 128-byte swizzle, rows past the valid ones read as zero).  The issuer runs a unit's k16 step 0
// (both accumulator groups) and commits, then step 1: the producers rewrite half h of the A stage
// for the next unit as soon as the MMAs of step h are done, from a slot that TMA filled while
// the previous MMAs ran.
constexpr int GM_RAW_HALF = TC_BM * 128;        // 16 KB: 128 rows x 16 words
constexpr int GM_RAW_ARR = 2 * GM_RAW_HALF;     // one operand's K chunk (32 words)

template <int MODE, bool TMA, int ND>
__global__ void __launch_bounds__((ND + GM_PROD + 1) * 32, 1)
k_gr_matmul_tc(const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1,
               const GrMMArgs a, unsigned* __restrict__ err, unsigned err_flag) {
  static_assert(!TMA || MODE != 2, "bit operands take the register path");
  constexpr int DC = 256 / ND;                              // columns per drain warp
  static_assert(ND == 8 || ND == 16, "drain warps");
  constexpr int NST = TMA ? 1 : NSTAGE;                     // A digit-plane stages
  constexpr int SLOT = (MODE == 1 ? 2 : 1) * GM_RAW_HALF;   // raw half-unit slot (TMA)
  constexpr int NSLOT = MODE == 1 ? 2 : 4;
  static_assert(!TMA || NSLOT * SLOT <= (NSTAGE - NST) * 8 * A_TILE, "raw slots");
  extern __shared__ unsigned char dsm[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  unsigned char* Bsm = base;                       // [2 chunks][8 planes][64 rows][64 B]
  unsigned char* Asm = base + 2 * GM_BCHUNK;       // [NST][8 planes][128 rows][64 B]
  unsigned char* Raw = Asm + NST * 8 * A_TILE;     // TMA: [NSLOT][SLOT]
  unsigned char* Osm = Asm + NSTAGE * 8 * A_TILE;  // [drain warp][32 rows][48 B]
  __shared__ __align__(8) u64 full_bar[NSTAGE], empty_bar[NSTAGE];
  __shared__ __align__(8) u64 raw_full[4], raw_empty[4], hfull[2], hempty[2];
  __shared__ __align__(8) u64 accf_bar[2], acce_bar[2], done_bar;
  __shared__ __align__(8) u64 stg_full, stg_free;
  __shared__ unsigned tmem_slot;
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;
  // bit-operand staging boxes (16 KB each, 1024-byte aligned) in the planes 1..7 of the A stages
  auto stg_box = [&](int b) -> unsigned char* {
    return Asm + (b < 3 ? (b + 1) * 16384 : 8 * A_TILE + 16384);
  };
  const bool out_tma = MODE == 2 && a.out_tma;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const long long R = a.R;
  const u64* p0 = a.p0;   // may alias out (a row is read before its tile is written)
  const u64* p1 = MODE == 1 ? a.p1 : nullptr;
  const u64 s1 = a.s1;
  constexpr int a_bits = MODE == 2 ? 1 : 0;
  // CTA b takes tiles b, b + G, b + 2G, ... (G = gridDim.x), or with matrix groups the
  // contiguous range [t0, t0 + count), so that it meets each matrix in one run
  const long long ntiles = (R + TC_BM - 1) / TC_BM;
  const long long G = gridDim.x;
  const bool contig = a.mrows != 0;
  const long long t0 = contig ? ntiles * blockIdx.x / G : blockIdx.x;
  const long long tstep = contig ? 1 : G;
  const long long count = contig ? ntiles * (blockIdx.x + 1) / G - t0
                                 : (ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / G + 1 : 0);
  const long long nunits = 2 * count;

  if (tid == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(&full_bar[i], GM_PROD);
      mbar_init(&empty_bar[i], 1);
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(&raw_full[i], 1);
      mbar_init(&raw_empty[i], GM_PROD);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&hfull[i], GM_PROD);
      mbar_init(&hempty[i], 1);
    }
    for (int g = 0; g < 2; ++g) {
      mbar_init(&accf_bar[g], 1);
      mbar_init(&acce_bar[g], ND);
    }
    mbar_init(&stg_full, ND);
    mbar_init(&stg_free, 1);
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;

  auto fail = [&]() {
    *abort = 1;
    atomicOr(err, err_flag);
  };

  if (warp >= ND && warp < ND + GM_PROD) {
    // ---- producers: B planes per matrix group, the A planes of every (tile, chunk) ----
    const int pt = tid - ND * 32;   // 0 .. 32 GM_PROD - 1
    const long long lda = a.in.s1;           // A row (bit word) stride inside a tile
    bool ok = true;
    long long cur_m = -1;
    // Before unit u is written: its stage must have been read by the MMAs of unit u - NSTAGE;
    // at a tile's first chunk, B is rebuilt when the matrix group changes (after the previous
    // tile's MMAs) and the next tile's rows are prefetched into L2.
    auto begin_unit = [&](long long u) -> bool {
      const int st = (int)(u % NST);
      if (u >= NST &&
          !__all_sync(0xffffffffu, mbar_wait(&empty_bar[st], (unsigned)(((u / NST) + 1) & 1), abort)))
        return false;
      if (u & 1) return true;
      const long long tile = t0 + (u >> 1) * tstep;
      const long long rho0 = tile * TC_BM;
      const long long mi = a.mrows ? rho0 / a.mrows : 0;
      if (mi != cur_m) {
        if (u > 0 && !__all_sync(0xffffffffu, mbar_wait(&empty_bar[(u - 1) % NST],
                                                         (unsigned)(((u - 1) / NST) & 1), abort)))
          return false;
        const u64* Mm = a.Mmat + mi * 4096;
        for (int it = pt; it < 64 * 8; it += GM_PROD * 32) {   // (row c of M^T, unit of 8 k)
          const int c = it >> 3, k8 = it & 7;
          u64 v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] = Mm[(k8 * 8 + q) * 64 + c];
          split8_store(v, Bsm + (k8 >> 2) * GM_BCHUNK, B_TILE, sw64_off(c, k8 & 3), a_bits != 0);
        }
        cur_m = mi;
        // the next group's matrix into L2 (this CTA's tiles are contiguous, so it comes next)
        if (pt == 0 && a.mrows && (mi + 1) * a.mrows < R) prefetch_l2(Mm + 4096, 4096 * 8);
      }
      if (!TMA && pt == 0 && (u >> 1) + 1 < count && lda <= 128) {   // next tile's rows into L2
        const long long r0 = (tile + tstep) * TC_BM;
        long long nr = (R - r0 < TC_BM) ? R - r0 : TC_BM;
        if (a.qvalid && a.qvalid - r0 % a.in.q < nr) nr = a.qvalid - r0 % a.in.q;
        const long long nb = rowmap(a.in, r0);
        const long long words = nr > 0 ? (nr - 1) * lda + (a_bits ? 1 : 64) : 0;
        const long long bytes = (words * 8) & ~15ll;   // whole 16-byte units inside the rows
        for (int w2 = 0; w2 < (p1 ? 2 : 1); ++w2) {
          const char* lo = reinterpret_cast<const char*>((w2 ? p1 : p0) + nb);
          for (long long o = 0; o < bytes; o += 65536)
            prefetch_l2(lo + o, (unsigned)(bytes - o < 65536 ? bytes - o : 65536));
        }
      }
      return true;
    };
    // rows of the tile at rho0 that exist (R, and the valid part of a padded segment)
    auto tile_rows = [&](long long rho0) -> long long {
      long long v = R - rho0;
      if (a.qvalid) {
        const long long rest = a.qvalid - rho0 % a.in.q;
        v = rest < v ? rest : v;
      }
      return v;
    };
    auto end_unit = [&](long long u) {
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_bar[u % NST]);
    };
    if constexpr (TMA) {
      // half-unit hu = 2u + h: K words 16 h .. 16 h + 15 of unit u (the items with u4 = 2h, 2h + 1).
      // One thread keeps NSLOT half-units of raw rows in flight; a slot is refilled once every
      // producer warp has split it.
      const bool tma_thr = pt == 0;
      const long long nhu = 2 * nunits;
      long long issued = 0, consumed = 0;
      auto issue_raw = [&](long long hu) {
        const int sl = (int)(hu % NSLOT);
        const long long u = hu >> 1;
        const long long rho0 = (t0 + (u >> 1) * tstep) * TC_BM;
        const int kx = (int)(u & 1) * 32 + (int)(hu & 1) * 16;
        const int y = (int)(a.in.q ? rho0 % a.in.q : rho0);
        const int z = (int)(a.in.q && a.in.s2 ? rho0 / a.in.q : 0);
        unsigned char* dst = Raw + sl * SLOT;
        mbar_expect_tx(&raw_full[sl], (unsigned)SLOT);
        tma_load_3d(dst, &tm0, &raw_full[sl], kx, y, z);
        if (MODE == 1) tma_load_3d(dst + GM_RAW_HALF, &tm1, &raw_full[sl], kx, y, z);
      };
      if (tma_thr)
        for (; issued < nhu && issued < NSLOT; ++issued) issue_raw(issued);
      constexpr int NIT = (256 + GM_PROD * 32 - 1) / (GM_PROD * 32);   // items per thread
      for (long long hu = 0; hu < nhu && ok; ++hu) {
        const long long u = hu >> 1;
        const int h = (int)(hu & 1);
        const int sl = (int)(hu % NSLOT);
        if (!(ok = __all_sync(0xffffffffu,
                              mbar_wait(&raw_full[sl], (unsigned)((hu / NSLOT) & 1), abort))))
          break;
        if (h == 0 && !(u & 1)) {
          // a tile's first half-unit: B is rebuilt when the matrix group changes, once every
          // MMA of the previous unit is done
          const long long tile = t0 + (u >> 1) * tstep;
          const long long mi = a.mrows ? tile * TC_BM / a.mrows : 0;
          if (mi != cur_m) {
            if (u > 0 && !(ok = __all_sync(0xffffffffu,
                                           mbar_wait(&hempty[1], (unsigned)((u - 1) & 1), abort))))
              break;
            const u64* Mm = a.Mmat + mi * 4096;
            for (int it = pt; it < 64 * 8; it += GM_PROD * 32) {   // (row c of M^T, unit of 8 k)
              const int c = it >> 3, k8 = it & 7;
              u64 v[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) v[q] = Mm[(k8 * 8 + q) * 64 + c];
              split8_store(v, Bsm + (k8 >> 2) * GM_BCHUNK, B_TILE, sw64_off(c, k8 & 3));
            }
            cur_m = mi;
            if (pt == 0 && a.mrows && (mi + 1) * a.mrows < R) prefetch_l2(Mm + 4096, 4096 * 8);
          }
        }
        // half h of the A stage is free once the MMAs of step h of unit u - 1 are done
        if (u > 0 && !(ok = __all_sync(0xffffffffu,
                                       mbar_wait(&hempty[h], (unsigned)((u - 1) & 1), abort))))
          break;
        const unsigned char* r0 = Raw + sl * SLOT;
#pragma unroll
        for (int q = 0; q < NIT; ++q) {
          // item = (row, unit of 8 k): the 8 lanes of a shared-memory phase take 8 consecutive
          // rows of one unit, conflict-free in the swizzled raw rows and in the digit planes
          const int item = pt + q * GM_PROD * 32;
          if (item < 256) {
            const int row = item & (TC_BM - 1), u4 = 2 * h + (item >> 7);
            const unsigned char* src = r0 + row * 128;
            u64 v[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int c = (((u4 & 1) * 4 + j) ^ (row & 7)) * 16;   // 128-byte swizzle
              const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(src + c);
              v[2 * j] = x.x;
              v[2 * j + 1] = x.y;
              if (MODE == 1) {
                const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(src + GM_RAW_HALF + c);
                v[2 * j] -= w.x;
                v[2 * j + 1] -= w.y;
              }
            }
            split8_store(v, Asm, A_TILE, sw64_off(row, u4));
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&hfull[h]);
          mbar_arrive(&raw_empty[sl]);
        }
        ++consumed;
        bool iok = true;
        if (tma_thr && issued < nhu) {
          iok = mbar_wait(&raw_empty[sl], (unsigned)((hu / NSLOT) & 1), abort);
          if (iok) issue_raw(issued++);
        }
        ok = __all_sync(0xffffffffu, iok);
      }
      // loads still in flight land before the CTA leaves
      if (tma_thr)
        for (long long hu = consumed; hu < issued; ++hu)
          mbar_wait_plain(&raw_full[hu % NSLOT], (unsigned)((hu / NSLOT) & 1));
    } else if (a_bits) {
      constexpr int NIT = (512 + GM_PROD * 32 - 1) / (GM_PROD * 32);   // items per thread
      // One bit word per row serves both K chunks of its tile (bytes 0..3, then 4..7); the
      // words of tile t + 1 are in flight while tile t's two chunks are written.
      auto load_tile = [&](long long t, u64 (&w)[NIT]) {
        const long long rho0 = (t0 + t * tstep) * TC_BM;
        const long long ib = rowmap(a.in, rho0);   // word index of the tile's first bit word
        const long long vrows = tile_rows(rho0);
#pragma unroll
        for (int q = 0; q < NIT; ++q) {
          const int item = pt + q * GM_PROD * 32;
          const bool in = item < 512 && (item >> 2) < vrows;
          w[q] = in ? p0[ib + (item >> 2) * lda] : 0ull;
        }
      };
      u64 wd[NIT], nd[NIT];
      if (count > 0) load_tile(0, nd);
      for (long long t = 0; t < count && ok; ++t) {
#pragma unroll
        for (int q = 0; q < NIT; ++q) wd[q] = nd[q];
        if (t + 1 < count) load_tile(t + 1, nd);
#pragma unroll 1
        for (int kc = 0; kc < 2; ++kc) {
          const long long u = 2 * t + kc;
          if (!(ok = begin_unit(u))) break;
          unsigned char* As = Asm + (u % NSTAGE) * 8 * A_TILE;
#pragma unroll
          for (int q = 0; q < NIT; ++q) {
            const int item = pt + q * GM_PROD * 32;
            if (item < 512) {
              const unsigned by = (unsigned)(wd[q] >> (kc * 32 + (item & 3) * 8)) & 0xFFu;
              *reinterpret_cast<uint4*>(As + sw64_off(item >> 2, item & 3)) = bits_plane0(by);
            }
          }
          end_unit(u);
        }
      }
    } else {
      // A rows in rounds of NQ items (8 words each) per thread, RPU rounds per unit; the loads
      // of round k + 1 are in flight while round k is split into the stage, across unit ends
      auto stream = [&](auto nqc, auto p1c) {
        constexpr int NQ = decltype(nqc)::value;
        constexpr bool P1 = decltype(p1c)::value;
        constexpr int RPU = (512 + NQ * GM_PROD * 32 - 1) / (NQ * GM_PROD * 32);
        const long long nrounds = nunits * RPU;
        u64 cv[NQ][8], nv[NQ][8], nw[NQ][8];   // current round (p0 - p1 formed), next round
        auto issue = [&](long long k, u64 (&v)[NQ][8], u64 (&w)[NQ][8]) {
          const long long u = k / RPU;
          const int r = (int)(k - u * RPU);
          const long long rho0 = (t0 + (u >> 1) * tstep) * TC_BM;
          const long long ib = rowmap(a.in, rho0) + (u & 1) * 32;
          const long long vrows = tile_rows(rho0);
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int item = pt + (r * NQ + q) * GM_PROD * 32;   // (row, unit of 8 k)
            const bool in = item < 512 && (item >> 2) < vrows;
            const long long off = ib + (item >> 2) * lda + (item & 3) * 8;
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
              const ulonglong2 x =
                  in ? *reinterpret_cast<const ulonglong2*>(p0 + off + j) : make_ulonglong2(0, 0);
              v[q][j] = x.x;
              v[q][j + 1] = x.y;
              if (P1) {
                const ulonglong2 y =
                    in ? *reinterpret_cast<const ulonglong2*>(p1 + off + j) : make_ulonglong2(0, 0);
                w[q][j] = y.x;
                w[q][j + 1] = y.y;
              }
            }
          }
        };
        // the next round becomes the current one (the subtraction waits for its loads)
        auto take_next = [&]() {
#pragma unroll
          for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int j = 0; j < 8; ++j) cv[q][j] = P1 ? nv[q][j] - nw[q][j] : nv[q][j];
        };
        if (nrounds > 0) {
          issue(0, nv, nw);
          take_next();
        }
        for (long long k = 0; k < nrounds; ++k) {
          const long long u = k / RPU;
          const int r = (int)(k - u * RPU);
          if (k + 1 < nrounds) issue(k + 1, nv, nw);
          if (r == 0 && !(ok = begin_unit(u))) break;
          unsigned char* As = Asm + (u % NSTAGE) * 8 * A_TILE;
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int item = pt + (r * NQ + q) * GM_PROD * 32;
            if (item < 512) split8_store(cv[q], As, A_TILE, sw64_off(item >> 2, item & 3));
          }
          if (r == RPU - 1) end_unit(u);
          if (k + 1 < nrounds) take_next();
        }
      };
      if (MODE == 1) stream(std::integral_constant<int, 2>(), std::true_type());
      else stream(std::integral_constant<int, 3>(), std::false_type());
    }
    if (!ok && lane == 0) fail();
  } else if (warp == ND + GM_PROD) {
    // ---- MMA issuer ----
    if (lane == 0 && TMA) {
      // per unit: k16 step 0 of both groups, commit (half 0 free), step 1, commit (half 1 free)
      const u64 ad = smem_desc(Asm, 64);
      const u64 db0 = smem_desc(Bsm, 64);
      for (long long u = 0; u < nunits; ++u) {
        const u64 bd = db0 + (u64)(((int)(u & 1) * GM_BCHUNK) >> 4);
        const bool first = !(u & 1), last = (u & 1) != 0;
        const long long v = u >> 1;
        const unsigned ph = (unsigned)(u & 1);
        if (!mbar_wait(&hfull[0], ph, abort)) { fail(); break; }
        tc_fence_after();
        if (first && v > 0 && !mbar_wait(&acce_bar[0], (unsigned)((v - 1) & 1), abort)) { fail(); break; }
        tc_fence_after();
        issue_group<0, false, 0>(tmem, ad, bd, first ? 1u : 0u);
        if (first && v > 0 && !mbar_wait(&acce_bar[1], (unsigned)((v - 1) & 1), abort)) { fail(); break; }
        tc_fence_after();
        issue_group<1, false, 0>(tmem, ad, bd, first ? 1u : 0u);
        mma_commit(&hempty[0]);
        if (!mbar_wait(&hfull[1], ph, abort)) { fail(); break; }
        tc_fence_after();
        issue_group<0, false, 1>(tmem, ad, bd, 0u);
        if (last) mma_commit(&accf_bar[0]);
        issue_group<1, false, 1>(tmem, ad, bd, 0u);
        if (last) mma_commit(&accf_bar[1]);
        mma_commit(&hempty[1]);
      }
      mma_commit(&done_bar);
      mbar_wait_plain(&done_bar, 0u);
    } else if (lane == 0) {
      const u64 da0 = smem_desc(Asm, 64);
      const u64 db0 = smem_desc(Bsm, 64);
      for (long long u = 0; u < nunits; ++u) {
        const int st = (int)(u % NST);
        if (!mbar_wait(&full_bar[st], (unsigned)((u / NST) & 1), abort)) { fail(); break; }
        tc_fence_after();
        const u64 ad = da0 + (u64)((st * 8 * A_TILE) >> 4);
        const u64 bd = db0 + (u64)(((int)(u & 1) * GM_BCHUNK) >> 4);
        // both K chunks of a tile go into one accumulation, drained once per tile
        const int kc = (int)(u & 1);
        const bool first = kc == 0, last = kc == 1;
        const long long v = u >> 1;   // accumulation (tile) index
        if (first && v > 0 && !mbar_wait(&acce_bar[0], (unsigned)((v - 1) & 1), abort)) { fail(); break; }
        tc_fence_after();
        if (a_bits) issue_group<0, true>(tmem, ad, bd, first ? 1u : 0u);
        else issue_group<0>(tmem, ad, bd, first ? 1u : 0u);
        if (last) mma_commit(&accf_bar[0]);
        if (first && v > 0 && !mbar_wait(&acce_bar[1], (unsigned)((v - 1) & 1), abort)) { fail(); break; }
        tc_fence_after();
        if (a_bits) issue_group<1, true>(tmem, ad, bd, first ? 1u : 0u);
        else issue_group<1>(tmem, ad, bd, first ? 1u : 0u);
        if (last) mma_commit(&accf_bar[1]);
        mma_commit(&empty_bar[st]);
      }
      mma_commit(&done_bar);
      mbar_wait_plain(&done_bar, 0u);
    }
  } else if (warp < ND) {
    // ---- drain warps: rows 32 (w % 4) + lane, columns DC (w / 4) .. +DC-1 ----
    const int q4 = warp & 3, h = warp >> 2;
    const unsigned tl = tmem + ((unsigned)(q4 * 32) << 16) + (unsigned)(h * DC);
    u64 acc[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) acc[c] = 0;
    bool ok = true;
    long long nst = 0;                   // tiles stored by TMA so far
    const long long nacc = nunits / 2;   // one accumulation per tile
    for (long long v = 0; v < nacc && ok; ++v) {
      const unsigned par = (unsigned)(v & 1);
      // the rows this lane stores in the two passes (16 rows per pass, 2 lanes per row) as word
      // offsets (-1: none) and their add0 offsets
      long long obr[2], rg[2];
      auto tile_rows_out = [&]() {
        const long long r = (t0 + v * tstep) * TC_BM + q4 * 32 + lane;   // this lane's row
        const bool exists = r < R && (!a.qvalid || r % a.in.q < a.qvalid);
        const long long ob = exists ? rowmap(a.om, r) : -1;
        const bool live = ob >= 0 && ob < a.out_lim;
        const long long ao =
            !a.add0 ? 0 : (a.add0_in ? (exists ? rowmap(a.in, r) : 0) : r * a.ld_add0);
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
          const int rr = pass * 16 + (lane >> 1);
          obr[pass] = __shfl_sync(0xffffffffu, live ? ob : -1, rr);
          rg[pass] = __shfl_sync(0xffffffffu, ao, rr);
        }
      };
      // add0 words of the stored 16-byte chunks: a fold has the first EARLY columns in flight
      // during the drains; the rows come before the drains except for bit operands
      constexpr int EARLY = MODE == 1 ? DC / 2 : 0;
      if (MODE != 2) tile_rows_out();
      ulonglong2 ad[DC / 4][2];
      auto load_add0 = [&](int c0) {
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
          const long long col = h * DC + c0 + 2 * (lane & 1);
          ad[c0 / 4][pass] = (a.add0 && obr[pass] >= 0)
                                 ? *reinterpret_cast<const ulonglong2*>(a.add0 + rg[pass] + col)
                                 : make_ulonglong2(0, 0);
        }
      };
#pragma unroll
      for (int c0 = 0; c0 < EARLY; c0 += 4) load_add0(c0);
#pragma unroll 1
      for (int g = 0; g < 2; ++g) {
        ok = __all_sync(0xffffffffu, mbar_wait(&accf_bar[g], par, abort));
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int c16 = 0; c16 < DC / 16; ++c16) {
          if (a_bits) {
            if (g == 0) drain16_pairs<0>(tl, c16 * 16, acc + c16 * 16);
            else drain16_pairs<1>(tl, c16 * 16, acc + c16 * 16);
          } else {
            if (g == 0) drain16<0>(tl, c16 * 16, acc + c16 * 16);
            else drain16<1>(tl, c16 * 16, acc + c16 * 16);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce_bar[g]);
      }
      // a bit-operand tile leaves by TMA stores when all its rows lie below the row limit
      // (uniform over the drain warps); the others take the register epilogue
      bool tile_tma = false;
      long long rho0 = 0;
      int ty = 0, tz = 0;
      if (out_tma) {
        rho0 = (t0 + v * tstep) * TC_BM;
        ty = (int)(a.om.q ? rho0 % a.om.q : rho0);
        tz = (int)(a.om.q ? rho0 / a.om.q : 0);
        const long long last = a.om.q ? ty + TC_BM - 1 : (rho0 + TC_BM - 1 < R ? rho0 + TC_BM - 1 : R - 1);
        const long long off = last * a.om.s1 + (long long)tz * a.om.s2;
        tile_tma = off + 64 <= a.out_lim;
      }
      if (ok && tile_tma) {   // tile complete: into the staging boxes, out by TMA stores
        const bool st_thr = warp == 0 && lane == 0;
        const unsigned spar = (unsigned)(nst & 1);
        if (st_thr) {
          if (nst > 0) bulk_wait_read0();   // the previous stores have read the boxes
          mbar_arrive(&stg_free);
        }
        ok = __all_sync(0xffffffffu, mbar_wait(&stg_free, spar, abort));
        if (ok) {
          const int r = q4 * 32 + lane;   // tile row
#pragma unroll
          for (int c = 0; c < DC; c += 2) {
            const int col = h * DC + c;   // word column
            const int k = (col & 15) >> 1;
            *reinterpret_cast<ulonglong2*>(stg_box(col >> 4) + r * 128 + ((k ^ (r & 7)) << 4)) =
                make_ulonglong2(acc[c], acc[c + 1]);
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&stg_full);
          bool sok = true;
          if (st_thr) {
            sok = mbar_wait(&stg_full, spar, abort);
            if (sok) {
#pragma unroll
              for (int b = 0; b < 4; ++b) tma_store_3d(&tm1, stg_box(b), 16 * b, ty, tz);
              bulk_commit();
            }
          }
          ok = __all_sync(0xffffffffu, sok);
        }
        ++nst;
#pragma unroll
        for (int c = 0; c < DC; ++c) acc[c] = 0;
      } else if (ok) {   // tile complete: add add0, store (4 columns at a time through shared memory)
        unsigned char* os = Osm + warp * GM_OSTAGE;
        if (MODE == 2) tile_rows_out();
#pragma unroll
        for (int c0 = EARLY; c0 < DC; c0 += 4) load_add0(c0);
#pragma unroll
        for (int c0 = 0; c0 < DC; c0 += 4) {
#pragma unroll
          for (int q = 0; q < 2; ++q)
            *reinterpret_cast<ulonglong2*>(os + lane * GM_OROW + q * 16) =
                make_ulonglong2(acc[c0 + 2 * q], acc[c0 + 2 * q + 1]);
          __syncwarp();
#pragma unroll
          for (int pass = 0; pass < 2; ++pass) {
            const int rr = pass * 16 + (lane >> 1), ch = lane & 1;
            ulonglong2 w = *reinterpret_cast<const ulonglong2*>(os + rr * GM_OROW + ch * 16);
            if (obr[pass] >= 0) {
              const long long col = h * DC + c0 + 2 * ch;
              w.x += ad[c0 / 4][pass].x;
              w.y += ad[c0 / 4][pass].y;
              *reinterpret_cast<ulonglong2*>(a.out + obr[pass] + col) = w;
            }
          }
          __syncwarp();
        }
#pragma unroll
        for (int c = 0; c < DC; ++c) acc[c] = 0;
      }
    }
    // the stores still in flight complete before the CTA leaves
    if (out_tma && warp == 0 && lane == 0) bulk_wait0();
    if (!ok && lane == 0) fail();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---- GR-matrix products with the A operand in tensor memory ------------------------------------
// The same product as k_gr_matmul_tc (plain and fold modes), laid out so that an MMA reads only B
// from shared memory.  With N = 64 fixed by the ring degree, an MMA whose A (4 KB) and B (2 KB)
// both come from shared memory is bound by shared-memory reads (48 cycles for 128 x 64 x 16);
// here A's eight digit planes (K = 64: 8 x 32 columns) sit in tensor memory next to the eight
// accumulators of one output half (8 x 32 columns), and the output is computed in two halves of
// 32 columns, each MMA 128 x 32 x 16 reading 1 KB of B.
//   - TMA loads a tile's raw A rows (and p1's in a fold) into shared memory (boxes of 16 words x
//     128 rows, 128-byte swizzle, rows past the valid ones as zero);
//   - four producer warps, one per tensor-memory lane quarter, take one row per thread: the
//     8-word units are split into digit planes and written with tcgen05.st into the A columns;
//   - the MMA thread issues, per tile, the four units (half h, accumulator group G) into the
//     group's columns once the drain of its previous use is done;
//   - eight drain warps (rows 32 (w % 4) + lane, 16 columns each) drain a unit, add add0 and
//     store the half through shared memory as in k_gr_matmul_tc.
// A tile's A columns are rewritten only after all of its MMAs have completed.
constexpr int TM_NDRAIN = 8, TM_NPROD = 4;
constexpr int TM_THREADS = (TM_NDRAIN + TM_NPROD + 1) * 32;   // 416
constexpr int TM_DC = 16;                                      // columns per drain warp and half
constexpr int TM_RAW_ARR = TC_BM * 64 * 8;                     // 64 KB: one operand's tile
constexpr unsigned TM_A_COL = 256;                             // A planes at columns 256 .. 511
// Instruction descriptor, kind::f16: f32 accumulator, f16 A and B, K-major, M = 128, N = 32.
constexpr unsigned IDESC_N32 = (1u << 4) | ((unsigned)(32 >> 3) << 17) | ((unsigned)(TC_BM >> 4) << 24);

__host__ __device__ constexpr int tm_acc_col(int s) {   // group A {0,1,6,7} then B {2,3,4,5}
  return s == 0 ? 0 : s == 1 ? 32 : s == 6 ? 64 : s == 7 ? 96 : 128 + (s - 2) * 32;
}
constexpr size_t tm_smem(int mode) {
  return (size_t)2 * GM_BCHUNK + (size_t)2 * TM_RAW_ARR + (size_t)TM_NDRAIN * GM_OSTAGE + 1024;
  (void)mode;
}

// D (+)= A B with A in tensor memory
__device__ __forceinline__ void mma_f16_ta(unsigned d_tmem, unsigned a_tmem, u64 bdesc,
                                           unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(IDESC_N32), "r"(acc));
}
__device__ __forceinline__ void tmem_st4(unsigned taddr, const unsigned v[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// 8 consecutive u64 values -> their 8 digit planes, 4 f16 pairs each (the split of split8_store)
__device__ __forceinline__ void split8_regs(const u64 v[8], unsigned pk[8][4]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const u64 a = v[2 * m] + 0x8080808080808080ull, b = v[2 * m + 1] + 0x8080808080808080ull;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned xa = (unsigned)(a >> (32 * h)), xb = (unsigned)(b >> (32 * h));
      const unsigned a02 = __byte_perm(xa, 0x64u, 0x4240), a13 = __byte_perm(xa, 0x64u, 0x4341);
      const unsigned b02 = __byte_perm(xb, 0x64u, 0x4240), b13 = __byte_perm(xb, 0x64u, 0x4341);
      pk[4 * h + 0][m] = f16x2_minus_1152(__byte_perm(a02, b02, 0x5410));
      pk[4 * h + 2][m] = f16x2_minus_1152(__byte_perm(a02, b02, 0x7632));
      pk[4 * h + 1][m] = f16x2_minus_1152(__byte_perm(a13, b13, 0x5410));
      pk[4 * h + 3][m] = f16x2_minus_1152(__byte_perm(a13, b13, 0x7632));
    }
  }
}

// The MMAs of accumulator group G for output half h: A from tensor memory (plane i at column
// TM_A_COL + 32 i, k at + k / 2), B plane j of K chunk kc at bd0 + kc GM_BCHUNK + j B_TILE, its
// rows 32 h .. 32 h + 31 (2 KB further per half), 16 of K per MMA.
template <int G>
__device__ __forceinline__ void tm_issue_group(unsigned tmem, u64 bd0, int h) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int s = group_s(G, g);
#pragma unroll
    for (int kc = 0; kc < 2; ++kc)
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (i <= s) {
            const unsigned at = tmem + TM_A_COL + (unsigned)(32 * i + 16 * kc + 8 * kk);
            const u64 bd = bd0 + (u64)((kc * GM_BCHUNK + (s - i) * B_TILE + h * 32 * 64) >> 4) +
                           (u64)(kk * 2);
            const bool first = kc == 0 && kk == 0 && i == 0;
            mma_f16_ta(tmem + (unsigned)tm_acc_col(s), at, bd, first ? 0u : 1u);
          }
        }
  }
}

// drain of group G for the 16 columns at tl (+ the group's accumulator columns): as drain16
template <int G>
__device__ __forceinline__ void tm_drain16(unsigned tl, u64* acc) {
  constexpr int s0 = G == 0 ? 0 : 2, s1 = G == 0 ? 6 : 4;
#pragma unroll
  for (int h8 = 0; h8 < 16; h8 += 8) {
    unsigned x0[8], x1[8], y0[8], y1[8];
    tmem_ld8(tl + (unsigned)(tm_acc_col(s0) + h8), x0);
    tmem_ld8(tl + (unsigned)(tm_acc_col(s0 + 1) + h8), x1);
    tmem_ld8(tl + (unsigned)(tm_acc_col(s1) + h8), y0);
    tmem_ld8(tl + (unsigned)(tm_acc_col(s1 + 1) + h8), y1);
    tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const unsigned ws =
          (unsigned)f2i_biased(x0[j]) + (unsigned)f2i_biased(x1[j]) * 256u - PAIR_BIAS;
      const unsigned whi = f32_int(y0[j]) + f32_int(y1[j]) * 256u;
      acc[h8 + j] += (G == 0 ? (u64)(long long)(int)ws : (u64)(long long)(int)ws << 16) +
                     ((u64)(G == 0 ? (whi << 16) : whi) << 32);
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(TM_THREADS, 1)
k_gr_matmul_tm(const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1,
               const GrMMArgs a, unsigned* __restrict__ err, unsigned err_flag) {
  static_assert(MODE == 0 || MODE == 1, "plain and fold modes");
  constexpr int NRAW = MODE == 1 ? 1 : 2;                    // raw tile buffers
  constexpr int RAW_TILE = (MODE == 1 ? 2 : 1) * TM_RAW_ARR;
  extern __shared__ unsigned char dsm[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  unsigned char* Bsm = base;                               // [2 chunks][8 planes][64 rows][64 B]
  unsigned char* Raw = base + 2 * GM_BCHUNK;               // [NRAW][RAW_TILE]
  unsigned char* Osm = Raw + 2 * TM_RAW_ARR;               // [drain warp][32 rows][48 B]
  __shared__ __align__(8) u64 raw_full[2], raw_empty[2], a_full, a_empty;
  __shared__ __align__(8) u64 accf_bar[2], acce_bar[2], done_bar;
  __shared__ unsigned tmem_slot;
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const long long R = a.R;
  const long long ntiles = (R + TC_BM - 1) / TC_BM;
  const long long G = gridDim.x;
  const bool contig = a.mrows != 0;
  const long long t0 = contig ? ntiles * blockIdx.x / G : blockIdx.x;
  const long long tstep = contig ? 1 : G;
  const long long count = contig ? ntiles * (blockIdx.x + 1) / G - t0
                                 : (ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / G + 1 : 0);

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&raw_full[i], 1);
      mbar_init(&raw_empty[i], TM_NPROD);
    }
    mbar_init(&a_full, TM_NPROD);
    mbar_init(&a_empty, 1);
    for (int g = 0; g < 2; ++g) {
      mbar_init(&accf_bar[g], 1);
      mbar_init(&acce_bar[g], TM_NDRAIN);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;

  auto fail = [&]() {
    *abort = 1;
    atomicOr(err, err_flag);
  };

  if (warp >= TM_NDRAIN && warp < TM_NDRAIN + TM_NPROD) {
    // ---- producers: row = 32 (warp % 4) + lane of every tile; B planes per matrix group ----
    const int pw = warp - TM_NDRAIN;                // 0 .. 3 = the warp's lane quarter
    const int pt = pw * 32 + lane;                  // 0 .. 127
    const int row = (warp & 3) * 32 + lane;         // tensor-memory lane of this thread
    const unsigned trow = tmem + ((unsigned)((warp & 3) * 32) << 16);
    const bool tma_thr = pt == 0;
    long long issued = 0, consumed = 0, cur_m = -1;
    bool ok = true;
    auto issue_raw = [&](long long v) {
      const int rb = (int)(v % NRAW);
      const long long rho0 = (t0 + v * tstep) * TC_BM;
      const int y = (int)(a.in.q ? rho0 % a.in.q : rho0);
      const int z = (int)(a.in.q && a.in.s2 ? rho0 / a.in.q : 0);
      unsigned char* dst = Raw + rb * RAW_TILE;
      mbar_expect_tx(&raw_full[rb], (unsigned)RAW_TILE);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        tma_load_3d(dst + b * GM_RAW_HALF, &tm0, &raw_full[rb], 16 * b, y, z);
        if (MODE == 1) tma_load_3d(dst + TM_RAW_ARR + b * GM_RAW_HALF, &tm1, &raw_full[rb], 16 * b, y, z);
      }
    };
    if (tma_thr)
      for (; issued < count && issued < NRAW; ++issued) issue_raw(issued);
    for (long long v = 0; v < count && ok; ++v) {
      const int rb = (int)(v % NRAW);
      if (!(ok = __all_sync(0xffffffffu, mbar_wait(&raw_full[rb], (unsigned)((v / NRAW) & 1), abort))))
        break;
      // every MMA of tile v - 1 has read A (and B)
      if (v > 0 && !(ok = __all_sync(0xffffffffu, mbar_wait(&a_empty, (unsigned)((v - 1) & 1), abort))))
        break;
      tc_fence_after();
      const long long rho0 = (t0 + v * tstep) * TC_BM;
      const long long mi = a.mrows ? rho0 / a.mrows : 0;
      if (mi != cur_m) {   // B = M^T of this row group, split into its digit planes
        const u64* Mm = a.Mmat + mi * 4096;
        for (int it = pt; it < 64 * 8; it += TM_NPROD * 32) {   // (row c of M^T, unit of 8 k)
          const int c = it >> 3, k8 = it & 7;
          u64 w[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) w[q] = Mm[(k8 * 8 + q) * 64 + c];
          split8_store(w, Bsm + (k8 >> 2) * GM_BCHUNK, B_TILE, sw64_off(c, k8 & 3));
        }
        fence_proxy_async_smem();
        cur_m = mi;
      }
      const unsigned char* src = Raw + rb * RAW_TILE + row * 128;
#pragma unroll 2
      for (int u4 = 0; u4 < 8; ++u4) {   // words 8 u4 .. 8 u4 + 7 of the row
        const unsigned char* s0 = src + (u4 >> 1) * GM_RAW_HALF;
        u64 x[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = (((u4 & 1) * 4 + j) ^ (row & 7)) * 16;   // 128-byte swizzle
          const ulonglong2 p = *reinterpret_cast<const ulonglong2*>(s0 + c);
          x[2 * j] = p.x;
          x[2 * j + 1] = p.y;
          if (MODE == 1) {
            const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(s0 + TM_RAW_ARR + c);
            x[2 * j] -= w.x;
            x[2 * j + 1] -= w.y;
          }
        }
        unsigned pk[8][4];
        split8_regs(x, pk);
#pragma unroll
        for (int p = 0; p < 8; ++p) tmem_st4(trow + TM_A_COL + (unsigned)(32 * p + 4 * u4), pk[p]);
      }
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&a_full);
        mbar_arrive(&raw_empty[rb]);
      }
      ++consumed;
      bool iok = true;
      if (tma_thr && issued < count) {
        iok = mbar_wait(&raw_empty[rb], (unsigned)((v / NRAW) & 1), abort);
        if (iok) issue_raw(issued++);
      }
      ok = __all_sync(0xffffffffu, iok);
    }
    if (tma_thr)
      for (long long v = consumed; v < issued; ++v)
        mbar_wait_plain(&raw_full[v % NRAW], (unsigned)((v / NRAW) & 1));
    if (!ok && lane == 0) fail();
  } else if (warp == TM_NDRAIN + TM_NPROD) {
    // ---- MMA issuer: per tile, units (h, G) in the order (0,0) (0,1) (1,0) (1,1) ----
    if (lane == 0) {
      const u64 db0 = smem_desc(Bsm, 64);
      bool ok = true;
      for (long long v = 0; v < count && ok; ++v) {
        if (!(ok = mbar_wait(&a_full, (unsigned)(v & 1), abort))) break;
        tc_fence_after();
        for (int h = 0; h < 2 && ok; ++h) {
          const long long q = 2 * v + h;   // use of each accumulator group
          for (int g = 0; g < 2; ++g) {
            if (q > 0 && !(ok = mbar_wait(&acce_bar[g], (unsigned)((q - 1) & 1), abort))) break;
            tc_fence_after();
            if (g == 0) tm_issue_group<0>(tmem, db0, h);
            else tm_issue_group<1>(tmem, db0, h);
            mma_commit(&accf_bar[g]);
          }
        }
        if (ok) mma_commit(&a_empty);
      }
      if (!ok) fail();
      mma_commit(&done_bar);
      mbar_wait_plain(&done_bar, 0u);
    }
  } else if (warp < TM_NDRAIN) {
    // ---- drain warps: rows 32 (w % 4) + lane, columns 16 (w / 4) of each half ----
    const int q4 = warp & 3, hw = warp >> 2;
    const unsigned tl = tmem + ((unsigned)(q4 * 32) << 16) + (unsigned)(hw * TM_DC);
    u64 acc[TM_DC];
    bool ok = true;
    for (long long v = 0; v < count && ok; ++v) {
      // the rows this lane stores in the two passes (16 rows per pass, 2 lanes per row) as word
      // offsets (-1: none) and their add0 offsets
      long long obr[2], rg[2];
      {
        const long long r = (t0 + v * tstep) * TC_BM + q4 * 32 + lane;
        const bool exists = r < R && (!a.qvalid || r % a.in.q < a.qvalid);
        const long long ob = exists ? rowmap(a.om, r) : -1;
        const bool live = ob >= 0 && ob < a.out_lim;
        const long long ao =
            !a.add0 ? 0 : (a.add0_in ? (exists ? rowmap(a.in, r) : 0) : r * a.ld_add0);
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
          const int rr = pass * 16 + (lane >> 1);
          obr[pass] = __shfl_sync(0xffffffffu, live ? ob : -1, rr);
          rg[pass] = __shfl_sync(0xffffffffu, ao, rr);
        }
      }
      for (int h = 0; h < 2 && ok; ++h) {
        const long long q = 2 * v + h;
        const int col0 = h * 32 + hw * TM_DC;   // first output column of this warp's slice
        ulonglong2 ad[TM_DC / 4][2];
#pragma unroll
        for (int c0 = 0; c0 < TM_DC; c0 += 4)
#pragma unroll
          for (int pass = 0; pass < 2; ++pass) {
            const long long col = col0 + c0 + 2 * (lane & 1);
            ad[c0 / 4][pass] = (a.add0 && obr[pass] >= 0)
                                   ? *reinterpret_cast<const ulonglong2*>(a.add0 + rg[pass] + col)
                                   : make_ulonglong2(0, 0);
          }
#pragma unroll
        for (int c = 0; c < TM_DC; ++c) acc[c] = 0;
#pragma unroll 1
        for (int g = 0; g < 2; ++g) {
          ok = __all_sync(0xffffffffu, mbar_wait(&accf_bar[g], (unsigned)(q & 1), abort));
          if (!ok) break;
          tc_fence_after();
          if (g == 0) tm_drain16<0>(tl, acc);
          else tm_drain16<1>(tl, acc);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acce_bar[g]);
        }
        if (!ok) break;
        unsigned char* os = Osm + warp * GM_OSTAGE;
#pragma unroll
        for (int c0 = 0; c0 < TM_DC; c0 += 4) {
#pragma unroll
          for (int qq = 0; qq < 2; ++qq)
            *reinterpret_cast<ulonglong2*>(os + lane * GM_OROW + qq * 16) =
                make_ulonglong2(acc[c0 + 2 * qq], acc[c0 + 2 * qq + 1]);
          __syncwarp();
#pragma unroll
          for (int pass = 0; pass < 2; ++pass) {
            const int rr = pass * 16 + (lane >> 1), ch = lane & 1;
            ulonglong2 w = *reinterpret_cast<const ulonglong2*>(os + rr * GM_OROW + ch * 16);
            if (obr[pass] >= 0) {
              const long long col = col0 + c0 + 2 * ch;
              w.x += ad[c0 / 4][pass].x;
              w.y += ad[c0 / 4][pass].y;
              *reinterpret_cast<ulonglong2*>(a.out + obr[pass] + col) = w;
            }
          }
          __syncwarp();
        }
      }
    }
    if (!ok && lane == 0) fail();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---- Gram sums of the dense Pi_Reduce rounds -------------------------------------------------
// For vectors u, v of n = 2 Dh GR elements (rows of 64 words, element i at row i) a job adds
//   P[ee] += s G(u_even, v_even), P[oo] += s G(u_odd, v_odd), P[x] += s (G(u_even, v_odd) + G(u_odd, v_even))
// with G(u, v)[a][b] = sum_i u_i[a] v_i[b] (each block a 64 x 64 matrix, mod 2^64) and s the job's
// sign; u = a0 + sa1 a1 and v = b0 + sb1 b1 (a1, b1 may be absent).  The MMA tile is M = 128
// (rows a: u_even coefficients, then u_odd) x N = 64 (v of one parity, blockIdx.y) with K = the
// element pairs i, split across blockIdx.x; blockIdx.z is the job; each CTA adds its partial tile
// atomically.  Producers combine and split the rows into digit planes transposed to K-major; MMA
// issue and drains as in k_limb_gemm_tc; the drain warps accumulate over all of the CTA's chunks.
constexpr size_t GR_SMEM = (size_t)NSTAGE * STAGE + 1024;   // 2 x (64 KB A + 32 KB B)

template <bool GEN>
__global__ void __launch_bounds__(GM_THREADS, 1)
k_gram_tc(long long Dh, const GramJobs jobs, unsigned* __restrict__ err, unsigned err_flag) {
  extern __shared__ unsigned char dsm[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) u64 full_bar[NSTAGE], empty_bar[NSTAGE];
  __shared__ __align__(8) u64 accf_bar[2], acce_bar[2], done_bar;
  __shared__ unsigned tmem_slot;
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;

  const GramJob& J = jobs.j[blockIdx.z];
  const u64* __restrict__ x = J.a0;
  const u64* __restrict__ y = J.b0;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int par = blockIdx.y;                      // parity of y in this CTA's tile
  const long long nch = (Dh + TC_BK - 1) / TC_BK;  // chunks of 32 element pairs
  const long long c0 = nch * blockIdx.x / gridDim.x;
  const long long c1 = nch * (blockIdx.x + 1) / gridDim.x;
  const long long nunits = c1 - c0;

  if (tid == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(&full_bar[i], GM_PROD);
      mbar_init(&empty_bar[i], 1);
    }
    for (int g = 0; g < 2; ++g) {
      mbar_init(&accf_bar[g], 1);
      mbar_init(&acce_bar[g], GM_NDRAIN);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;

  auto fail = [&]() {
    *abort = 1;
    atomicOr(err, err_flag);
  };

  if (warp >= GM_NDRAIN && warp < GM_NDRAIN + GM_PROD) {
    // ---- producers: 512 A items (x rows a = item % 128, 8 pairs k8 = item / 128) and 256 B
    // items (y rows b = item % 64, k8 = item / 64), lanes on consecutive coefficients ----
    const int pt = tid - GM_NDRAIN * 32;
    constexpr int NITEM = 768;
    // rounds of NQ items per thread, RPU rounds per unit; the loads of round k + 1 are in flight
    // while round k is split into the stage, across unit ends
    // (one item per round with a second source, whose words need registers of their own)
    constexpr int NQ = GEN ? 1 : 2;
    constexpr int NQ2 = GEN ? NQ : 1;
    constexpr int RPU = (NITEM + NQ * GM_PROD * 32 - 1) / (NQ * GM_PROD * 32);
    const long long nrounds = nunits * RPU;
    bool ok = true;
    u64 cv[NQ][8], nv[NQ][8];
    u64 cv2[NQ2][8], nv2[NQ2][8];
    const u64* __restrict__ x1 = GEN ? J.a1 : nullptr;
    const u64* __restrict__ y1 = GEN ? J.b1 : nullptr;
    auto issue = [&](long long k, u64 (&v)[NQ][8], u64 (&v2)[NQ2][8]) {
      const long long u = k / RPU;
      const int r = (int)(k - u * RPU);
      const long long i0 = (c0 + u) * TC_BK;   // first element pair of the chunk
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int item = pt + (r * NQ + q) * GM_PROD * 32;
        const bool isA = item < 512;
        const int it = isA ? item : item - 512;
        const int row = isA ? (it & 127) : (it & 63);
        const int k8 = isA ? (it >> 7) : (it >> 6);
        // A row a: coefficient a % 64 of x_{2i + a / 64}; B row b: coefficient b of y_{2i + par}
        const long long roff = isA ? (row >> 6) * 64 + (row & 63) : par * 64 + row;
        const u64* src = (isA ? x : y) + roff;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const long long i = i0 + k8 * 8 + j;
          v[q][j] = (item < NITEM && i < Dh) ? src[i * 128] : 0ull;
        }
        if (GEN) {
          const u64* s2 = isA ? x1 : y1;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const long long i = i0 + k8 * 8 + j;
            v2[q][j] = (s2 && item < NITEM && i < Dh) ? s2[roff + i * 128] : 0ull;
          }
        }
      }
    };
    if (nrounds > 0) issue(0, cv, cv2);
    for (long long k = 0; k < nrounds; ++k) {
      const long long u = k / RPU;
      const int r = (int)(k - u * RPU);
      const int st = (int)(u % NSTAGE);
      if (k + 1 < nrounds) issue(k + 1, nv, nv2);
      if (r == 0) {
        if (u >= NSTAGE &&
            !(ok = __all_sync(0xffffffffu,
                              mbar_wait(&empty_bar[st], (unsigned)(((u / NSTAGE) + 1) & 1), abort))))
          break;
        const long long i1 = (c0 + u + 1) * TC_BK;
        if (pt == 0 && u + 1 < nunits) {   // next chunk's 32 pairs (64 rows) of x and y
          const long long np = (Dh - i1 < TC_BK) ? Dh - i1 : TC_BK;
          if (np > 0) {
            prefetch_l2(x + i1 * 128, (unsigned)(np * 1024));
            prefetch_l2(y + i1 * 128, (unsigned)(np * 1024));
          }
        }
      }
      unsigned char* As = base + st * STAGE;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int item = pt + (r * NQ + q) * GM_PROD * 32;
        if (item < NITEM) {
          const bool isA = item < 512;
          const int it = isA ? item : item - 512;
          unsigned char* dst = isA ? As : As + 8 * A_TILE;
          const int off = isA ? sw64_off(it & 127, it >> 7) : sw64_off(it & 63, it >> 6);
          if (GEN) {
            const u64 sc = isA ? J.sa1 : J.sb1;
#pragma unroll
            for (int j = 0; j < 8; ++j) cv[q][j] += sc * cv2[q][j];
          }
          split8_store(cv[q], dst, isA ? A_TILE : B_TILE, off);
        }
      }
      if (r == RPU - 1) {
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full_bar[st]);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          cv[q][j] = nv[q][j];
          if (GEN) cv2[q][j] = nv2[q][j];
        }
    }
    if (!ok && lane == 0) fail();
  } else if (warp == GM_NDRAIN + GM_PROD) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const u64 d0 = smem_desc(base, 64);
      for (long long u = 0; u < nunits; ++u) {
        const int st = (int)(u % NSTAGE);
        if (!mbar_wait(&full_bar[st], (unsigned)((u / NSTAGE) & 1), abort)) { fail(); break; }
        tc_fence_after();
        const u64 ad = d0 + (u64)((st * STAGE) >> 4);
        const u64 bd = ad + (u64)((8 * A_TILE) >> 4);
        // accumulation v takes chunks 2v and 2v + 1 (64 element pairs)
        const bool first = !(u & 1), last = (u & 1) || u == nunits - 1;
        const long long v = u >> 1;
        if (first && v > 0 && !mbar_wait(&acce_bar[0], (unsigned)((v - 1) & 1), abort)) { fail(); break; }
        tc_fence_after();
        issue_group<0>(tmem, ad, bd, first ? 1u : 0u);
        if (last) mma_commit(&accf_bar[0]);
        if (first && v > 0 && !mbar_wait(&acce_bar[1], (unsigned)((v - 1) & 1), abort)) { fail(); break; }
        tc_fence_after();
        issue_group<1>(tmem, ad, bd, first ? 1u : 0u);
        if (last) mma_commit(&accf_bar[1]);
        mma_commit(&empty_bar[st]);
      }
      mma_commit(&done_bar);
      mbar_wait_plain(&done_bar, 0u);
    }
  } else if (warp < GM_NDRAIN) {
    // ---- drain warps: tile rows 32 (w % 4) + lane, columns GM_DC (w / 4) .. +GM_DC-1 ----
    const int q4 = warp & 3, h = warp >> 2;
    const unsigned tl = tmem + ((unsigned)(q4 * 32) << 16) + (unsigned)(h * GM_DC);
    u64 acc[GM_DC];
#pragma unroll
    for (int c = 0; c < GM_DC; ++c) acc[c] = 0;
    bool ok = true;
    const long long nacc = (nunits + 1) / 2;
    for (long long v = 0; v < nacc && ok; ++v) {
      const unsigned pv = (unsigned)(v & 1);
#pragma unroll 1
      for (int g = 0; g < 2; ++g) {
        ok = __all_sync(0xffffffffu, mbar_wait(&accf_bar[g], pv, abort));
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int c16 = 0; c16 < GM_DC / 16; ++c16) {
          if (g == 0) drain16<0>(tl, c16 * 16, acc + c16 * 16);
          else drain16<1>(tl, c16 * 16, acc + c16 * 16);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce_bar[g]);
      }
    }
    if (ok && !*abort && nunits > 0) {
      const int a = q4 * 32 + lane;                // tile row: x parity a / 64, coefficient a % 64
      const int xpar = a >> 6;
      // (x parity, y parity) -> P block: (0,0) -> ee, (1,1) -> oo, mixed -> cross
      const long long blk = xpar != par ? jobs.off_x : (xpar ? jobs.off_oo : 0);
      u64* dst = J.P + blk + (a & 63) * 64 + h * GM_DC;
      const u64 sg = J.sign;
#pragma unroll
      for (int c = 0; c < GM_DC; ++c)
        atomicAdd(reinterpret_cast<unsigned long long*>(dst + c), (unsigned long long)(sg * acc[c]));
    } else if (!ok && lane == 0) {
      fail();
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace

size_t limb_tc_scratch_bytes(long long M, long long N, long long K, int nterms) {
  const long long Kp = ((nterms * K + TC_BK - 1) / TC_BK) * TC_BK;
  const long long a = 8 * M * Kp * 2, b = 8 * N * Kp * 2;
  return (size_t)(((a + 255) & ~255ll) + ((b + 255) & ~255ll) + 256);
}

int limb_gemm_tc(cudaStream_t st, long long M, long long N, long long K, int nterms,
                 const GemmTerm* terms, const Epi& epi, void* scratch, unsigned* err,
                 unsigned err_flag, cudaEvent_t ev0, cudaEvent_t ev1, int split_min) {
  if (M <= 0 || N <= 0) return 0;
  if (epi.atomic) return -1;
  const long long Kp = ((nterms * K + TC_BK - 1) / TC_BK) * TC_BK;
  unsigned short* Ap = reinterpret_cast<unsigned short*>(scratch);
  const long long abytes = (8 * M * Kp * 2 + 255) & ~255ll;
  unsigned short* Bp = reinterpret_cast<unsigned short*>(reinterpret_cast<char*>(scratch) + abytes);
  GemmTerm t1 = nterms > 1 ? terms[1] : terms[0];
  const int tpb = 256;
  long long ga = (M * (Kp / 8) + tpb - 1) / tpb, gb = (N * (Kp / 8) + tpb - 1) / tpb;
  if (ga > (1 << 20)) ga = 1 << 20;
  if (gb > (1 << 20)) gb = 1 << 20;
  k_split_digits<<<(unsigned)ga, tpb, 0, st>>>(terms[0], t1, nterms, 0, M, K, Kp, Ap);
  if (terms[0].B.trans == 0 && t1.B.trans == 0 && (Kp + 63) / 64 <= 65535) {
    dim3 g2((unsigned)((N + 31) / 32), (unsigned)((Kp + 63) / 64));
    k_split_digits_bt<<<g2, 256, 0, st>>>(terms[0], t1, nterms, N, K, Kp, Bp);
  } else {
    k_split_digits<<<(unsigned)gb, tpb, 0, st>>>(terms[0], t1, nterms, 1, N, K, Kp, Bp);
  }
  CUtensorMap ma, mb;
  if (!make_map(&ma, Ap, M, Kp, TC_BM) || !make_map(&mb, Bp, N, Kp, TC_BN)) return -2;
  const size_t smem = (size_t)NSTAGE * STAGE + (size_t)NDRAIN * 32 * 48 + 1024;
  set_max_dynamic_smem(reinterpret_cast<const void*>(k_limb_gemm_tc), (int)smem);
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
  }
  const long long tiles = ((M + TC_BM - 1) / TC_BM) * ((N + TC_BN - 1) / TC_BN);
  const long long nch = Kp / TC_BK;
  // thin products: split K (at least split_min chunks each) while the CTAs still fit one wave
  if (split_min <= 0) split_min = 8;
  long long nsplit = 1;
  while (tiles * nsplit * 2 <= nsm && nch / (nsplit * 2) >= split_min) nsplit *= 2;
  if (nsplit > 1) cudaMemset2DAsync(epi.out, (size_t)epi.ldc * 8, 0, (size_t)N * 8, (size_t)M, st);
  dim3 grid((unsigned)((M + TC_BM - 1) / TC_BM), (unsigned)((N + TC_BN - 1) / TC_BN),
            (unsigned)nsplit);
  if (ev0) cudaEventRecord(ev0, st);
  k_limb_gemm_tc<<<grid, TC_THREADS, smem, st>>>(ma, mb, M, N, Kp, epi.out, epi.ldc, err, err_flag);
  if (ev1) cudaEventRecord(ev1, st);
  long long ge = ((M * N + 7) / 8 + 255) / 256;
  if (ge > (1 << 20)) ge = 1 << 20;
  if (ge < 1) ge = 1;
  k_apply_epilogue<<<(unsigned)ge, 256, 0, st>>>(M, N, epi);
  return 0;
}

// Tensor map of the A rows of a GR-matrix product for the TMA producers: element (k, y, z) is
// word k of row y of block z, at base + y s1 + z s2 words (rows y < the valid ones; the rest read
// as zero).  Row maps with q = 0 are one block of R rows; with q > 0 a block of q rows (only the
// first qvalid exist when qvalid > 0), blocks s2 words apart (one block when s2 = 0: the rows
// repeat).  Boxes of 16 words x 128 rows, 128-byte swizzle.  false: not expressible (the caller
// takes the register path).
bool make_rows_map(CUtensorMap* map, const u64* base, const GrRowMap& in, long long R,
                   long long qvalid) {
  auto enc = encode_fn();
  if (!enc || !base || in.s1 <= 0 || (in.s1 & 1) || (in.s2 & 1) || in.s2 < 0 ||
      (reinterpret_cast<uintptr_t>(base) & 15))
    return false;
  cuuint64_t dims[3], strides[2];
  dims[0] = 64;
  if (in.q == 0) {
    dims[1] = (cuuint64_t)R;
    dims[2] = 1;
  } else {
    if (in.s2 && R % in.q) return false;   // a ragged last block would read past its rows
    dims[1] = (cuuint64_t)(qvalid > 0 ? qvalid : in.q);
    dims[2] = in.s2 ? (cuuint64_t)(R / in.q) : 1;
  }
  strides[0] = (cuuint64_t)in.s1 * 8;
  strides[1] = in.s2 ? (cuuint64_t)in.s2 * 8 : dims[1] * strides[0];
  if (dims[1] == 0 || dims[1] >= (1ull << 31) || dims[2] >= (1ull << 31)) return false;
  cuuint32_t box[3] = {16, (cuuint32_t)TC_BM, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<u64*>(base), dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int gr_matmul_tc_ex(cudaStream_t st, const GrMMArgs& args, unsigned* err, unsigned err_flag) {
  GrMMArgs a = args;
  if (a.R <= 0) return 0;
  if (a.add0 && !a.ld_add0) a.ld_add0 = 64;
  if (a.p1 && a.s1 != ~0ull) return -1;   // the kernel forms p0 - p1 only
  auto odd = [](long long v) { return (v & 1) != 0; };
  const bool bad_in = !a.a_bits && (odd(a.in.s1) || odd(a.in.s2));
  // 16-byte vector accesses need even word offsets; a tile must not straddle a map period or
  // a matrix group
  if ((a.qvalid && !a.in.q) || (a.add0_in && (a.a_bits || a.qvalid < 0))) return -1;
  if (bad_in || odd(a.om.s1) || odd(a.om.s2) || (a.add0 && odd(a.ld_add0)) ||
      (a.in.q % TC_BM) || (a.om.q % TC_BM) || (a.mrows % TC_BM) || a.in.q < 0 || a.om.q < 0 ||
      a.mrows < 0 ||
      ((reinterpret_cast<uintptr_t>(a.p0) | reinterpret_cast<uintptr_t>(a.p1) |
        reinterpret_cast<uintptr_t>(a.add0) | reinterpret_cast<uintptr_t>(a.out)) & 15))
    return -1;
  if (a.out_lim <= 0) a.out_lim = LLONG_MAX;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
  }
  const long long ntiles = (a.R + TC_BM - 1) / TC_BM;
  const unsigned grid = (unsigned)(ntiles < nsm ? ntiles : nsm);
  const int mode = a.a_bits ? 2 : (a.p1 ? 1 : 0);
  CUtensorMap m0, m1;
  std::memset(&m0, 0, sizeof(m0));
  std::memset(&m1, 0, sizeof(m1));
  const bool tma = a.tma && mode != 2 && make_rows_map(&m0, a.p0, a.in, a.R, a.qvalid) &&
                   (mode == 0 || make_rows_map(&m1, a.p1, a.in, a.R, a.qvalid));
  // bit-operand tiles can leave by TMA stores when the output map covers exactly the rows that
  // exist: no padded segments, whole periods (the map then clips only rows past R); tiles with
  // rows at or past out_lim keep the register epilogue
  a.out_tma = 0;
  if (mode == 2 && a.tma && !a.qvalid && (a.om.q == 0 || (a.om.s2 != 0 && a.R % a.om.q == 0)))
    a.out_tma = make_rows_map(&m1, a.out, a.om, a.R, 0) ? 1 : 0;
  if (a.tma == 2 && mode != 2 && tma) {   // A operand in tensor memory
    const size_t smem = tm_smem(mode);
    auto launch_tm = [&](auto kern) {
      set_max_dynamic_smem(reinterpret_cast<const void*>(kern), (int)smem);
      kern<<<grid, TM_THREADS, smem, st>>>(m0, m1, a, err, err_flag);
    };
    if (mode == 1) launch_tm(k_gr_matmul_tm<1>);
    else launch_tm(k_gr_matmul_tm<0>);
    return 0;
  }
  const int nd = a.drain_warps == 16 ? 16 : 8;
  const size_t smem = (size_t)2 * GM_BCHUNK + (size_t)NSTAGE * 8 * A_TILE +
                      (size_t)nd * GM_OSTAGE + 1024;
  auto launch = [&](auto kern) {
    set_max_dynamic_smem(reinterpret_cast<const void*>(kern), (int)smem);
    kern<<<grid, (nd + GM_PROD + 1) * 32, smem, st>>>(m0, m1, a, err, err_flag);
  };
  if (nd == 16) {
    if (mode == 2) launch(k_gr_matmul_tc<2, false, 16>);
    else if (mode == 1 && tma) launch(k_gr_matmul_tc<1, true, 16>);
    else if (mode == 1) launch(k_gr_matmul_tc<1, false, 16>);
    else if (tma) launch(k_gr_matmul_tc<0, true, 16>);
    else launch(k_gr_matmul_tc<0, false, 16>);
  } else {
    if (mode == 2) launch(k_gr_matmul_tc<2, false, 8>);
    else if (mode == 1 && tma) launch(k_gr_matmul_tc<1, true, 8>);
    else if (mode == 1) launch(k_gr_matmul_tc<1, false, 8>);
    else if (tma) launch(k_gr_matmul_tc<0, true, 8>);
    else launch(k_gr_matmul_tc<0, false, 8>);
  }
  return 0;
}

int gram_jobs_tc(cudaStream_t st, long long Dh, const GramJobs& jobs, unsigned* err,
                 unsigned err_flag, int nsplit) {
  if (Dh <= 0 || jobs.n <= 0) return 0;
  if (jobs.n > GRAM_JOBS_MAX) return -1;
  // single-source jobs run in the kernel that keeps two items in flight per producer thread,
  // jobs with a second source in the one that holds both sources' words
  GramJobs one{}, two{};
  one.off_oo = two.off_oo = jobs.off_oo;
  one.off_x = two.off_x = jobs.off_x;
  for (int q = 0; q < jobs.n; ++q) {
    const GramJob& J = jobs.j[q];
    if (!J.a0 || !J.b0 || !J.P) return -1;
    if ((reinterpret_cast<uintptr_t>(J.a0) | reinterpret_cast<uintptr_t>(J.b0) |
         reinterpret_cast<uintptr_t>(J.a1) | reinterpret_cast<uintptr_t>(J.b1)) & 15)
      return -1;
    GramJobs& dst = (J.a1 || J.b1) ? two : one;
    dst.j[dst.n++] = J;
  }
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
  }
  const long long nch = (Dh + TC_BK - 1) / TC_BK;
  // CTAs per job and parity: nsplit (nsm / 2 by default) shared by the jobs of a launch
  auto grid_of = [&](int n) {
    long long split = nsplit > 0 ? nsplit : nsm / 2;
    split /= n;
    if (split > nch) split = nch;
    if (split < 1) split = 1;
    return dim3((unsigned)split, 2, (unsigned)n);
  };
  if (one.n) {
    set_max_dynamic_smem(reinterpret_cast<const void*>(k_gram_tc<false>), (int)GR_SMEM);
    k_gram_tc<false><<<grid_of(one.n), GM_THREADS, GR_SMEM, st>>>(Dh, one, err, err_flag);
  }
  if (two.n) {
    set_max_dynamic_smem(reinterpret_cast<const void*>(k_gram_tc<true>), (int)GR_SMEM);
    k_gram_tc<true><<<grid_of(two.n), GM_THREADS, GR_SMEM, st>>>(Dh, two, err, err_flag);
  }
  return 0;
}

int gram3_tc(cudaStream_t st, long long Dh, const u64* x, const u64* y, u64* P, unsigned* err,
             unsigned err_flag, int nsplit) {
  GramJobs jobs{};
  jobs.n = 1;
  jobs.off_oo = 4096;
  jobs.off_x = 2 * 4096;
  jobs.j[0] = GramJob{x, nullptr, 0ull, y, nullptr, 0ull, P, 1ull};
  return gram_jobs_tc(st, Dh, jobs, err, err_flag, nsplit);
}

}  // namespace mpc3
