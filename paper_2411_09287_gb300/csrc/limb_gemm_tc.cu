// Exact Z_2^64 GEMM on the 5th-generation tensor cores (tcgen05, kind::f16 with bf16 inputs,
// f32 accumulators in tensor memory): the "limb tensor-core path" of the local products of
// Pi_Inner (Fig. DPP, Sec. 4.1).
//
// Each u64 operand value is split into 8 balanced signed digits d_0..d_7 in [-128, 127] with
// v = sum_i 2^(8i) d_i mod 2^64 (carry-propagating split; the carry out of d_7 vanishes mod 2^64).
// bf16 holds every such digit exactly.  Only digit pairs with i + j < 8 contribute mod 2^64:
//   C = sum_{s<8} 2^(8s) C_s,   C_s = sum_{i+j=s} A_i B_j.
// C_s lives in its own TMEM accumulator (8 x 64 columns = all 512).  Within one K chunk of 64,
// |C_s| <= 8 * 64 * 2^14 = 2^23 < 2^24, so every f32 partial sum is an exact integer; after each
// chunk the accumulators are read back (tcgen05.ld), converted to integers and added, shifted by
// 8s, into 64-bit registers, which wrap mod 2^64 as required.
//
// Data flow per CTA (128 x 64 output tile, 128 threads):
//   - thread 0 loads the 8 + 8 digit-plane tiles of a K chunk with TMA (128B swizzle) and
//     issues the 36 x 4 MMAs (M = 128, N = 64, K = 16) in s-major order, then commits to an
//     mbarrier;
//   - all 4 warps wait on that mbarrier, drain their 32 TMEM lanes (= rows) and accumulate.
// Every mbarrier wait is bounded (clock64); on a timeout the CTA records an error in *err, waits
// (bounded) for its TMA copies, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "kernels.h"

namespace mpc3 {

namespace {

constexpr int TC_BM = 128, TC_BN = 64, TC_BK = 64;
constexpr int A_TILE = TC_BM * TC_BK * 2;   // 16 KB per digit plane
constexpr int B_TILE = TC_BN * TC_BK * 2;   // 8 KB per digit plane
constexpr unsigned TX_BYTES = 8 * (A_TILE + B_TILE);
constexpr long long WAIT_CYCLES = 2000000000ll;   // about one second at 2 GHz

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(u64* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(u64* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(u64* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, u64* bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<u64>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 bytes
// apart (the layout TMA writes for a box whose inner extent is 128 bytes).
__device__ __forceinline__ u64 smem_desc(const void* p) {
  const u64 addr = smem_u32(p);
  u64 d = 0;
  d |= (addr & 0x3FFFFull) >> 4;            // start address
  d |= (u64)(16 >> 4) << 16;                // leading byte offset (unused with swizzle)
  d |= (u64)(1024 >> 4) << 32;              // stride byte offset
  d |= (u64)1 << 46;                        // descriptor version
  d |= (u64)2 << 61;                        // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: f32 accumulator, bf16 A and B, both K-major, M = 128, N = 64.
constexpr unsigned IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TC_BN >> 3) << 17) |
                           ((unsigned)(TC_BM >> 4) << 24);

__device__ __forceinline__ void mma_f16(unsigned d_tmem, u64 adesc, u64 bdesc, unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float v[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(128, 1)
k_limb_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               long long M, long long N, long long Kp, u64* __restrict__ C, long long ldc,
               unsigned* __restrict__ err, unsigned err_flag) {
  extern __shared__ unsigned char dsm[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  unsigned char* As = base;                       // 8 x 16 KB
  unsigned char* Bs = base + 8 * A_TILE;          // 8 x 8 KB
  __shared__ __align__(8) u64 full_bar, mma_bar;
  __shared__ unsigned tmem_slot;
  __shared__ int abort_flag;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const long long m0 = (long long)blockIdx.x * TC_BM;
  const long long n0 = (long long)blockIdx.y * TC_BN;

  if (tid == 0) {
    mbar_init(&full_bar, 1);
    mbar_init(&mma_bar, 1);
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

  u64 acc[TC_BN];
#pragma unroll
  for (int c = 0; c < TC_BN; ++c) acc[c] = 0;

  const int nchunks = (int)(Kp / TC_BK);
  int stuck = 0;   // thread 0: 1 = TMA copies of the current chunk may be in flight, 2 = MMAs
  unsigned stuck_parity = 0;
  for (int ch = 0; ch < nchunks; ++ch) {
    const unsigned parity = (unsigned)(ch & 1);
    if (tid == 0) {
      mbar_expect_tx(&full_bar, TX_BYTES);
      const int kx = ch * TC_BK;
#pragma unroll 1
      for (int i = 0; i < 8; ++i) {
        tma_load_3d(As + i * A_TILE, &tmA, &full_bar, kx, (int)m0, i);
        tma_load_3d(Bs + i * B_TILE, &tmB, &full_bar, kx, (int)n0, i);
      }
      if (!mbar_wait_bounded(&full_bar, parity)) {
        abort_flag = 1;
        stuck = 1;
        stuck_parity = parity;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // s-major: accumulator s collects the digit pairs i + j = s; the first MMA of each
        // accumulator in a chunk overwrites it
#pragma unroll 1
        for (int s = 0; s < 8; ++s) {
#pragma unroll 1
          for (int kk = 0; kk < TC_BK / 16; ++kk) {
#pragma unroll 1
            for (int i = 0; i <= s; ++i) {
              const int j = s - i;
              const u64 ad = smem_desc(As + i * A_TILE) + (u64)(kk * 2);   // +32 bytes per k16
              const u64 bd = smem_desc(Bs + j * B_TILE) + (u64)(kk * 2);
              mma_f16(tmem + (unsigned)(s * TC_BN), ad, bd, (kk > 0 || i > 0) ? 1u : 0u);
            }
          }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&mma_bar))
            : "memory");
      }
    }
    __syncthreads();
    if (abort_flag) break;
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&mma_bar, parity));
    if (!ok) {
      abort_flag = 1;
      if (tid == 0) { stuck = 2; stuck_parity = parity; }
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const unsigned lane_base = (unsigned)(warp * 32) << 16;
#pragma unroll
      for (int s = 0; s < 8; ++s) {
#pragma unroll
        for (int c16 = 0; c16 < TC_BN / 16; ++c16) {
          float v[16];
          tmem_ld16(tmem + lane_base + (unsigned)(s * TC_BN + c16 * 16), v);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int q = 0; q < 16; ++q)
            acc[c16 * 16 + q] += (u64)__float2ll_rn(v[q]) << (8 * s);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (abort_flag) break;
  }

  if (abort_flag) {
    if (tid == 0) {
      atomicOr(err, err_flag);
      // let the copies or MMAs of the failed chunk finish before the memory is released
      if (stuck == 1) mbar_wait_bounded(&full_bar, stuck_parity);
      if (stuck == 2) mbar_wait_bounded(&mma_bar, stuck_parity);
    }
  } else {
    const long long r = m0 + warp * 32 + lane;
    if (r < M) {
#pragma unroll
      for (int c = 0; c < TC_BN; ++c)
        if (n0 + c < N) C[r * ldc + n0 + c] = acc[c];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
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

__device__ __forceinline__ void balanced_digits(u64 v, int d[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int b = (int)(v & 0xFFull);
    v >>= 8;
    if (b >= 128) {
      b -= 256;
      v += 1;
    }
    d[i] = b;
  }
}

__device__ __forceinline__ unsigned bf16_bits(int d) {   // exact for |d| <= 256
  return __float_as_uint((float)d) >> 16;
}

// planes[i][row][k'] (bf16), row-major with pitch Kp; element (row, k') of the concatenated
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
    unsigned packed[8][4];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const long long kk = kc * 8 + q;
      u64 v = 0;
      if (kk < (long long)nterms * K) {
        const GemmTerm& T = (kk < K) ? t0 : t1;
        const long long k = kk < K ? kk : kk - K;
        v = which ? load_opnd(T.B, k, row, K, R) : load_opnd(T.A, row, k, R, K);
      }
      int d[8];
      balanced_digits(v, d);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const unsigned b = bf16_bits(d[i]);
        if (q & 1) packed[i][q >> 1] |= b << 16;
        else packed[i][q >> 1] = b;
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      uint4 o;
      o.x = packed[i][0]; o.y = packed[i][1]; o.z = packed[i][2]; o.w = packed[i][3];
      *reinterpret_cast<uint4*>(planes + ((long long)i * R + row) * Kp + kc * 8) = o;
    }
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

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* map, void* planes, long long rows, long long Kp, int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, 8};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(rows * Kp * 2)};
  cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, planes, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

size_t limb_tc_scratch_bytes(long long M, long long N, long long K, int nterms) {
  const long long Kp = ((nterms * K + TC_BK - 1) / TC_BK) * TC_BK;
  const long long a = 8 * M * Kp * 2, b = 8 * N * Kp * 2;
  return (size_t)(((a + 255) & ~255ll) + ((b + 255) & ~255ll) + 256);
}

int limb_gemm_tc(cudaStream_t st, long long M, long long N, long long K, int nterms,
                 const GemmTerm* terms, const Epi& epi, void* scratch, unsigned* err,
                 unsigned err_flag) {
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
  k_split_digits<<<(unsigned)gb, tpb, 0, st>>>(terms[0], t1, nterms, 1, N, K, Kp, Bp);
  CUtensorMap ma, mb;
  if (!make_map(&ma, Ap, M, Kp, TC_BM) || !make_map(&mb, Bp, N, Kp, TC_BN)) return -2;
  const size_t smem = 8 * (A_TILE + B_TILE) + 1024;
  cudaFuncSetAttribute(k_limb_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((unsigned)((M + TC_BM - 1) / TC_BM), (unsigned)((N + TC_BN - 1) / TC_BN));
  k_limb_gemm_tc<<<grid, 128, smem, st>>>(ma, mb, M, N, Kp, epi.out, epi.ldc, err, err_flag);
  long long ge = ((M * N + 7) / 8 + 255) / 256;
  if (ge > (1 << 20)) ge = 1 << 20;
  if (ge < 1) ge = 1;
  k_apply_epilogue<<<(unsigned)ge, 256, 0, st>>>(M, N, epi);
  return 0;
}

}  // namespace mpc3
