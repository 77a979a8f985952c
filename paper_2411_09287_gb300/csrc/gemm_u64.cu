// Exact Z_2^64 GEMM on CUDA cores (the plain "u64 path").
//
// Computes C = sum_t A_t B_t mod 2^64 with operands formed on load (value = scale*(p0 + s1*p1)),
// which lets one kernel evaluate every local product of Pi_Inner (Fig. DPP, Sec. 4.1):
//   P0 : (R_X1 + R_X2)(R_W1 + R_W2)                       (offline Gamma)
//   P1 : M_X [R_W]_1 + [R_X]_1 M_W                          (online, negated in the epilogue)
//   P2 : M_X (M_W - [R_W]_2) - [R_X]_2 M_W                   (online)
// and, with split-K and atomic accumulation, the Gram sums sum_i u_i (x) v_i and the GR folds of
// the batched verification.  Tiles: BM x BN per CTA, BK = 8, TM x TN register micro-tiles,
// double-buffered shared memory.  Index arithmetic is 64-bit; every global access is bounds
// checked (out-of-range operand elements read as 0).
#include "kernels.h"

namespace mpc3 {

namespace {

__device__ __forceinline__ u64 ld_opnd(const Opnd& o, long long r, long long c, long long R,
                                       long long C) {
  if (r >= R || c >= C) return 0;
  if (o.trans == 2) {
    // bit-product operand of the truncation batch: row r = 64 j + j', column c = output e,
    // value = bit j of p0[e] AND bit j' of p1[e]
    return (o.p0[c] >> (r >> 6)) & (o.p1[c] >> (r & 63)) & 1ull;
  }
  const long long off = o.trans ? (c * o.ld + r) : (r * o.ld + c);
  u64 v = o.p0[off];
  if (o.p1) {   // the coefficients used are +-1: avoid the 3-IMAD u64 multiply for them
    const u64 w = o.p1[off];
    v = (o.s1 == 1ull) ? v + w : ((o.s1 == ~0ull) ? v - w : v + o.s1 * w);
  }
  if (o.scale != 1ull) v = (o.scale == ~0ull) ? (0ull - v) : o.scale * v;
  return v;
}

// The tile (bx, by) of split bz; a kernel body shared by the plain and the batched launches.
template <int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void gemm_u64_body(long long M, long long N, long long K, int nterms,
                                              const GemmTerm& t0, const GemmTerm& t1,
                                              const Epi& epi, long long k_per_split,
                                              long long bx, long long by, long long bz) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int A_PER = BM * BK / NT;
  constexpr int B_PER = BK * BN / NT;
  static_assert(BM * BK % NT == 0 && BK * BN % NT == 0, "tile/thread mismatch");
  __shared__ u64 As[2][BK][BM];
  __shared__ u64 Bs[2][BK][BN];

  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN);
  const int ty = tid / (BN / TN);
  const long long m0 = bx * BM;
  const long long n0 = by * BN;
  const long long kbeg = bz * k_per_split;
  const long long kend = (kbeg + k_per_split < K) ? (kbeg + k_per_split) : K;

  u64 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0;

  // virtual K loop over the terms: for term t, k runs over [kbeg, kend)
  const long long ktiles_per_term = (kend > kbeg) ? (kend - kbeg + BK - 1) / BK : 0;
  const long long total_tiles = ktiles_per_term * nterms;

  u64 ra[A_PER], rb[B_PER];
  auto load_tile = [&](long long tile) {
    const GemmTerm& T = (tile < ktiles_per_term) ? t0 : t1;
    const long long kt = kbeg + (tile % (ktiles_per_term ? ktiles_per_term : 1)) * BK;
#pragma unroll
    for (int q = 0; q < A_PER; ++q) {
      const int e = tid + q * NT;
      int mm, kk;
      if (T.A.trans == 1) { mm = e % BM; kk = e / BM; }  // consecutive threads: consecutive m
      else { kk = e % BK; mm = e / BK; }                  // consecutive threads: consecutive k
      const long long gk = kt + kk;
      ra[q] = (gk < kend) ? ld_opnd(T.A, m0 + mm, gk, M, K) : 0;
    }
#pragma unroll
    for (int q = 0; q < B_PER; ++q) {
      const int e = tid + q * NT;
      const int nn = e % BN, kk = e / BN;
      const long long gk = kt + kk;
      rb[q] = (gk < kend) ? ld_opnd(T.B, gk, n0 + nn, K, N) : 0;
    }
  };
  auto store_tile = [&](int buf, long long tile) {
    const GemmTerm& T = (tile < ktiles_per_term) ? t0 : t1;
#pragma unroll
    for (int q = 0; q < A_PER; ++q) {
      const int e = tid + q * NT;
      int mm, kk;
      if (T.A.trans == 1) { mm = e % BM; kk = e / BM; }
      else { kk = e % BK; mm = e / BK; }
      As[buf][kk][mm] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < B_PER; ++q) {
      const int e = tid + q * NT;
      Bs[buf][e / BN][e % BN] = rb[q];
    }
  };

  if (total_tiles > 0) {
    load_tile(0);
    store_tile(0, 0);
    __syncthreads();
    for (long long tile = 0; tile < total_tiles; ++tile) {
      const int buf = (int)(tile & 1);
      if (tile + 1 < total_tiles) load_tile(tile + 1);
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        u64 a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[buf][k][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[buf][k][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
      }
      if (tile + 1 < total_tiles) store_tile(buf ^ 1, tile + 1);
      __syncthreads();
    }
  }

  // epilogue
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const long long r = m0 + ty * TM + i;
    if (r >= M) continue;
    const long long cbase = n0 + tx * TN;
    u64 prfw[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) prfw[j] = 0;
    if (!epi.atomic && epi.prf_sign) {
      const long long ibase = r * epi.ldc + cbase;
      if ((TN % 8 == 0) && (ibase % 8 == 0)) {
#pragma unroll
        for (int j8 = 0; j8 < TN; j8 += 8) {
          u64 w[8];
          prf_block8(epi.key, epi.tag, epi.obj, (u64)(ibase + j8) >> 3, w);
#pragma unroll
          for (int q = 0; q < 8; ++q) prfw[j8 + q] = w[q];
        }
      } else {
#pragma unroll
        for (int j = 0; j < TN; ++j)
          if (cbase + j < N) prfw[j] = prf_word(epi.key, epi.tag, epi.obj, (u64)(ibase + j));
      }
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const long long c = cbase + j;
      if (c >= N) continue;
      const long long idx = r * epi.ldc + c;
      const u64 v = (epi.acc_sign == 1ull) ? acc[i][j]
                  : ((epi.acc_sign == ~0ull) ? 0ull - acc[i][j] : epi.acc_sign * acc[i][j]);
      if (epi.atomic) {
        atomicAdd(reinterpret_cast<unsigned long long*>(epi.out + idx), v);
      } else {
        u64 o = v;
        if (epi.add0) o += epi.add0[epi.ld_add0 ? r * epi.ld_add0 + c : idx];
        if (epi.add1) o += epi.add1[idx];
        o += epi.prf_sign * prfw[j];
        epi.out[idx] = o;
      }
    }
  }
}

template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_u64_kernel(long long M, long long N, long long K, int nterms, GemmTerm t0, GemmTerm t1,
                Epi epi, long long k_per_split) {
  gemm_u64_body<BM, BN, BK, TM, TN>(M, N, K, nterms, t0, t1, epi, k_per_split, blockIdx.x,
                                    blockIdx.y, blockIdx.z);
}

// Independent 64 x 64 Gram sums (one term each, atomic epilogues) in one launch: grid.y picks
// the sum.
struct GramBatchArgs {
  GemmTerm T[GRAM_BATCH_MAX];
  Epi e[GRAM_BATCH_MAX];
};
__global__ void __launch_bounds__(256)
gemm_u64_gram_batch_kernel(long long K, GramBatchArgs b, long long k_per_split) {
  const int t = blockIdx.y;
  gemm_u64_body<64, 64, 8, 4, 4>(64, 64, K, 1, b.T[t], b.T[t], b.e[t], k_per_split, 0, 0,
                                 blockIdx.z);
}

}  // namespace

void gemm_u64_gram_batch(cudaStream_t st, long long K, int n, const GemmTerm* terms,
                         const Epi* epis, int nsplit) {
  if (n <= 0 || K <= 0) return;
  if (nsplit < 1) nsplit = 1;
  GramBatchArgs b;
  for (int i = 0; i < n && i < GRAM_BATCH_MAX; ++i) {
    b.T[i] = terms[i];
    b.e[i] = epis[i];
  }
  const long long kps = (K + nsplit - 1) / nsplit;
  dim3 grid(1, (unsigned)(n < GRAM_BATCH_MAX ? n : GRAM_BATCH_MAX), (unsigned)nsplit);
  gemm_u64_gram_batch_kernel<<<grid, 256, 0, st>>>(K, b, kps);
}

void gemm_u64(cudaStream_t st, long long M, long long N, long long K, int nterms,
              const GemmTerm* terms, const Epi& epi, int nsplit) {
  if (M <= 0 || N <= 0) return;
  if (nsplit < 1) nsplit = 1;
  const long long kps = (K + nsplit - 1) / nsplit;
  GemmTerm t1 = (nterms > 1) ? terms[1] : terms[0];
  if (M <= 64 && N <= 64) {   // Gram sums (64 x 64 outputs, long K)
    constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4;
    dim3 grid(1, 1, (unsigned)nsplit);
    gemm_u64_kernel<BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(
        M, N, K, nterms, terms[0], t1, epi, kps);
  } else if (N <= 64) {
    constexpr int BM = 128, BN = 64, BK = 8, TM = 8, TN = 4;
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)nsplit);
    gemm_u64_kernel<BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(
        M, N, K, nterms, terms[0], t1, epi, kps);
  } else {
    constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)nsplit);
    gemm_u64_kernel<BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(
        M, N, K, nterms, terms[0], t1, epi, kps);
  }
}

void gemm_u64_small(cudaStream_t st, long long M, long long N, long long K, int nterms,
                    const GemmTerm* terms, const Epi& epi) {
  if (M <= 0 || N <= 0) return;
  constexpr int BM = 16, BN = 16, BK = 16, TM = 1, TN = 1;
  GemmTerm t1 = (nterms > 1) ? terms[1] : terms[0];
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), 1);
  gemm_u64_kernel<BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(
      M, N, K, nterms, terms[0], t1, epi, K);
}

}  // namespace mpc3
