// The matrix S_{j,j'} = sum_e r^(2e) b1_{e,j} b2_{e,j'} of the truncation-pair batch on the
// 5th-generation tensor cores (tcgen05.mma kind::f8f6f4, e4m3 operands, f32 accumulators in
// tensor memory), exactly.
//
// Why: in the consolidated trunc-pair claim (index i = 64 e + j), P0's cross-term sums of the first
// six Pi_Reduce rounds (Fig. Reduce) are all linear combinations of S with public GR weights, so
// S is computed once per layer.  Writing r^(2e) = T_hi[e_hi] T_lo[e_lo] with e = e_hi L + e_lo:
//   S_hi[e_hi][(j,j')] = sum_{e_lo} T_lo[e_lo] b1_{e,j} b2_{e,j'}     (this file, tensor cores)
//   S[(j,j')]          = sum_{e_hi} T_hi[e_hi] (x) S_hi[e_hi][(j,j')]  (a u64 GEMM + fold)
// Exactness: each u64 coefficient of T_lo is split into 16 unsigned 4-bit limbs; every limb value
// 0..15 and every bit 0/1 is exact in e4m3, and an accumulator sums at most L <= 2^16 terms of at
// most 15, so every f32 partial sum is an exact integer below 2^20; the limbs are recombined
// mod 2^64 when the e_lo loop ends.
//
// Operands, both K-major (K = e):
//   A (M = 128 pairs per accumulator): byte (p, e) = e4m3(b1_{e,j} AND b2_{e,j'}), generated in
//     shared memory by four warps from bit-transposed words BT[j][e / 64] (bit e % 64);
//   B (N = 256 limb columns): TL8[c][e_lo] = e4m3(limb c % 16 of coefficient c / 16 of T_lo[e_lo]),
//     loaded by TMA (128-byte swizzle).
// CTA = 256 pairs (j = 4 blockIdx.x .. +3, all j') x 256 limb columns (16 coefficients) x one e_hi
// block; two accumulators (pairs 0..127 and 128..255 of the tile) fill the 512 TMEM columns.
// Warps 0-3 generate A and drain TMEM at the end, warp 4 issues the TMA loads, warp 5 the MMAs;
// a 3-stage ring of 64 KB (two A tiles + one B tile per stage) keeps the three roles apart.
// Every mbarrier wait is bounded; a failure sets err_flag in *err and the CTA lets its copies and
// MMAs finish (bounded), frees its tensor memory and returns without writing.
#include "kernels.h"
#include "tcgen05.cuh"

namespace mpc3 {

namespace {

using namespace tc;

constexpr int S_KC = 128;                  // e per chunk (one 128-byte swizzled row)
constexpr int S_TPAIRS = 256;              // pairs per CTA (two accumulators of 128)
constexpr int S_TCOLS = 256;               // limb columns per CTA (16 coefficients x 16 limbs)
constexpr int S_ATILE = 128 * S_KC;        // 16 KB
constexpr int S_BTILE = S_TCOLS * S_KC;    // 32 KB
constexpr int S_STAGE = 2 * S_ATILE + S_BTILE;
constexpr int S_NST = 3;
constexpr int S_THREADS = 6 * 32;
constexpr size_t S_SMEM = (size_t)S_NST * S_STAGE + 1024;

// kind::f8f6f4: f32 accumulator, e4m3 A and B (format 0), both K-major, M = 128, N = 256
constexpr unsigned S_IDESC = (1u << 4) | ((unsigned)(S_TCOLS >> 3) << 17) | ((unsigned)(128 >> 4) << 24);

template <int ACC>
__device__ __forceinline__ void mma_f8(unsigned d_tmem, u64 adesc, u64 bdesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(S_IDESC), "n"(ACC));
}

// 4 bits -> 4 bytes of e4m3 1.0 (0x38) or 0: the multiply spreads bit b to byte b (no carries)
__device__ __forceinline__ unsigned nibble_bytes(unsigned nib) {
  return ((nib * 0x00204081u) & 0x01010101u) * 0x38u;
}

// e4m3 encodings of the integers 0..15
__device__ __constant__ unsigned char E4M3_INT[16] = {0x00, 0x38, 0x40, 0x44, 0x48, 0x4A, 0x4C, 0x4E,
                                                      0x50, 0x51, 0x52, 0x53, 0x54, 0x55, 0x56, 0x57};

// TL8[c * L + e] = e4m3(limb c % 16 of coefficient c / 16 of T_lo[e]), c < 1024, e < L.
// Each thread produces 16 consecutive e of one column (one 16-byte store).
__global__ void k_limb_table(const u64* __restrict__ Tlo, long long L, unsigned char* __restrict__ TL8) {
  const long long chunks = L / 16;
  const long long total = 1024 * chunks;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
       w += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(w / chunks);
    const long long e0 = (w % chunks) * 16;
    const int coeff = c >> 4, limb = c & 15;
    unsigned v[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const unsigned nib = (unsigned)((Tlo[(e0 + i) * 64 + coeff] >> (4 * limb)) & 15ull);
      v[i >> 2] |= (unsigned)E4M3_INT[nib] << (8 * (i & 3));
    }
    uint4 out;
    out.x = v[0]; out.y = v[1]; out.z = v[2]; out.w = v[3];
    *reinterpret_cast<uint4*>(TL8 + (long long)c * L + e0) = out;
  }
}

// BT[j * (Epad / 64) + w] = bits j of words[64 w .. 64 w + 63] (bit i = word 64 w + i).
// One 64-thread block per word group w: thread j gathers its bit of the 64 words.
__global__ void k_bit_transpose(const u64* __restrict__ words, long long nw, u64* __restrict__ BT) {
  __shared__ u64 wsh[64];
  for (long long w = blockIdx.x; w < nw; w += gridDim.x) {
    wsh[threadIdx.x] = words[w * 64 + threadIdx.x];
    __syncthreads();
    const int j = threadIdx.x;
    u64 v = 0;
#pragma unroll 8
    for (int i = 0; i < 64; ++i) v |= ((wsh[i] >> j) & 1ull) << i;
    BT[(long long)j * nw + w] = v;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(S_THREADS, 1)
k_trunc_s_tc(const __grid_constant__ CUtensorMap tmB, const u64* __restrict__ B1T,
             const u64* __restrict__ B2T, long long nw, long long L, u64* __restrict__ S_hi,
             unsigned* __restrict__ err, unsigned err_flag) {
  extern __shared__ unsigned char dsm[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) u64 fullb[S_NST], fulla[S_NST], empty[S_NST], done_bar;
  __shared__ unsigned tmem_slot;
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int pt = blockIdx.x, ct = blockIdx.y;
  const long long ehi = blockIdx.z;
  const int nchunks = (int)(L / S_KC);

  if (tid == 0) {
    for (int i = 0; i < S_NST; ++i) {
      mbar_init(&fullb[i], 1);
      mbar_init(&fulla[i], 4);
      mbar_init(&empty[i], 1);
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

  if (warp == 4) {
    // ---- TMA producer: limb-table tile (256 columns x 128 e) per chunk ----
    if (lane == 0) {
      int last = -1;
      for (int c = 0; c < nchunks; ++c) {
        const int st = c % S_NST;
        if (c >= S_NST && !mbar_wait(&empty[st], (unsigned)(((c / S_NST) + 1) & 1), abort)) {
          fail();
          break;
        }
        mbar_expect_tx(&fullb[st], (unsigned)S_BTILE);
        tma_load_2d(base + st * S_STAGE + 2 * S_ATILE, &tmB, &fullb[st], c * S_KC, ct * S_TCOLS);
        last = c;
      }
      for (int c = last; c >= 0 && c > last - S_NST; --c)
        mbar_wait_plain(&fullb[c % S_NST], (unsigned)((c / S_NST) & 1));
    }
  } else if (warp == 5) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const u64 d0 = smem_desc(base, 128);
      for (int c = 0; c < nchunks; ++c) {
        const int st = c % S_NST;
        const unsigned par = (unsigned)((c / S_NST) & 1);
        if (!mbar_wait(&fullb[st], par, abort) || !mbar_wait(&fulla[st], par, abort)) {
          fail();
          break;
        }
        tc_fence_after();
        const u64 ds = d0 + (u64)((st * S_STAGE) >> 4);
        const u64 db = ds + (u64)((2 * S_ATILE) >> 4);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const u64 da = ds + (u64)((a * S_ATILE) >> 4);
#pragma unroll
          for (int k = 0; k < S_KC / 32; ++k) {
            if (c == 0 && k == 0) mma_f8<0>(tmem + (unsigned)(a * 256), da + 2 * k, db + 2 * k);
            else mma_f8<1>(tmem + (unsigned)(a * 256), da + 2 * k, db + 2 * k);
          }
        }
        mma_commit(&empty[st]);
      }
      mma_commit(&done_bar);
      mbar_wait_plain(&done_bar, 0u);
    }
  } else {
    // ---- A generators (warps 0-3), then the drain ----
    const int jp = tid & 63, jj = tid >> 6;          // row tid of both tiles: j' and j offset
    const u64* b2row = B2T + (long long)jp * nw;
    const u64* b1row0 = B1T + (long long)(4 * pt + jj) * nw;
    const u64* b1row1 = B1T + (long long)(4 * pt + 2 + jj) * nw;
    const int r7 = tid & 7;
    const int roff = (tid >> 3) * 1024 + r7 * 128;
    const long long w0 = ehi * (L / 64);
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int st = c % S_NST;
      if (c >= S_NST) {
        ok = __all_sync(0xffffffffu, mbar_wait(&empty[st], (unsigned)(((c / S_NST) + 1) & 1), abort));
        if (!ok) break;
      }
      const long long w = w0 + 2 * c;
      const u64 m2lo = b2row[w], m2hi = b2row[w + 1];
      const u64 m[2][2] = {{b1row0[w] & m2lo, b1row0[w + 1] & m2hi},
                           {b1row1[w] & m2lo, b1row1[w + 1] & m2hi}};
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        unsigned char* row = base + st * S_STAGE + a * S_ATILE + roff;
#pragma unroll
        for (int q = 0; q < 8; ++q) {             // 16 e per 16-byte chunk, swizzled position
          const unsigned bits = (unsigned)(m[a][q >> 2] >> (16 * (q & 3))) & 0xFFFFu;
          uint4 v;
          v.x = nibble_bytes(bits & 15u);
          v.y = nibble_bytes((bits >> 4) & 15u);
          v.z = nibble_bytes((bits >> 8) & 15u);
          v.w = nibble_bytes(bits >> 12);
          *reinterpret_cast<uint4*>(row + ((q ^ r7) << 4)) = v;
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&fulla[st]);
    }
    if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&done_bar, 0u, abort));
    if (ok && !*abort) {
      tc_fence_after();
      const unsigned tl = tmem + ((unsigned)(warp * 32) << 16);
#pragma unroll 1
      for (int a = 0; a < 2; ++a) {
        const long long pair = (long long)pt * S_TPAIRS + a * 128 + warp * 32 + lane;
        u64* out = S_hi + (ehi * 4096 + pair) * 64 + ct * 16;
#pragma unroll 1
        for (int cc = 0; cc < 16; ++cc) {
          unsigned v[16];
          tmem_ld16(tl + (unsigned)(a * 256 + cc * 16), v);
          tmem_ld_wait();
          u64 sum = 0;
#pragma unroll
          for (int l = 0; l < 16; ++l)   // exact: 0 <= limb sum < 2^23, + 2^23 keeps it integral
            sum += (u64)(__float_as_uint(__uint_as_float(v[l]) + 8388608.0f) - 0x4B000000u) << (4 * l);
          out[cc] = sum;
        }
      }
    } else if (!ok && lane == 0) {
      fail();
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// out[p][c] = reduce(sum_{a+b=s} P[a*ld + p*64 + b]) for n pairs.
__global__ void k_fold_reduce_strided(const u64* __restrict__ P, long long ld, u64* __restrict__ out) {
  __shared__ u64 prod[128];
  const long long p = blockIdx.x;
  const int s = threadIdx.x;
  u64 v = 0;
  if (s < 127) {
    const int a0 = (s < 64) ? 0 : s - 63;
    const int a1 = (s < 64) ? s : 63;
    for (int a = a0; a <= a1; ++a) v += P[a * ld + p * 64 + (s - a)];
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
    out[p * 64 + s] = r;
  }
}

}  // namespace

void launch_trunc_limb_table(cudaStream_t st, const u64* Tlo, long long L, unsigned char* TL8) {
  const long long total = 1024 * (L / 16);
  long long g = (total + 255) / 256;
  if (g > (1ll << 20)) g = 1ll << 20;
  k_limb_table<<<(unsigned)g, 256, 0, st>>>(Tlo, L, TL8);
}

void launch_trunc_bit_transpose(cudaStream_t st, const u64* words, long long Epad, u64* BT) {
  const long long nw = Epad / 64;
  const long long g = nw < (1ll << 20) ? nw : (1ll << 20);
  k_bit_transpose<<<(unsigned)g, 64, 0, st>>>(words, nw, BT);
}

int launch_trunc_s_tc(cudaStream_t st, const u64* B1T, const u64* B2T, long long Epad,
                      const unsigned char* TL8, long long L, long long nhi, u64* S_hi,
                      unsigned* err, unsigned err_flag) {
  auto enc = encode_fn();
  if (!enc || L % S_KC != 0) return -2;
  CUtensorMap mb;
  cuuint64_t dims[2] = {(cuuint64_t)L, 1024};
  cuuint64_t strides[1] = {(cuuint64_t)L};
  cuuint32_t box[2] = {(cuuint32_t)S_KC, (cuuint32_t)S_TCOLS};
  cuuint32_t es[2] = {1, 1};
  if (enc(&mb, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<unsigned char*>(TL8), dims, strides,
          box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return -2;
  set_max_dynamic_smem(reinterpret_cast<const void*>(k_trunc_s_tc), (int)S_SMEM);
  dim3 grid(4096 / S_TPAIRS, 1024 / S_TCOLS, (unsigned)nhi);
  k_trunc_s_tc<<<grid, S_THREADS, S_SMEM, st>>>(mb, B1T, B2T, Epad / 64, L, S_hi, err, err_flag);
  return 0;
}

void launch_fold_reduce_strided(cudaStream_t st, const u64* P, long long ld, int npairs, u64* out) {
  k_fold_reduce_strided<<<npairs, 128, 0, st>>>(P, ld, out);
}

}  // namespace mpc3
