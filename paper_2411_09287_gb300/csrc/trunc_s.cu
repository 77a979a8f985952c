// The matrix S_{j,j'} = sum_e r^(2e) b1_{e,j} b2_{e,j'} of the truncation-pair batch on the tensor
// cores (legacy mma.sync, e4m3 inputs, f32 accumulation), exactly.
//
// Why: in the consolidated trunc-pair claim (index i = 64 e + j), P0's cross-term sums of the first
// six Pi_Reduce rounds (Fig. Reduce) are all linear combinations of S with public GR weights, so
// S is computed once per layer.  Writing r^(2e) = T_hi[e_hi] T_lo[e_lo] with e = e_hi L + e_lo:
//   S_hi[e_hi][(j,j')] = sum_{e_lo} T_lo[e_lo] b1_{e,j} b2_{e,j'}     (this file, tensor cores)
//   S[(j,j')]          = sum_{e_hi} T_hi[e_hi] (x) S_hi[e_hi][(j,j')]  (a u64 GEMM + fold)
// Exactness: each u64 coefficient of T_lo is split into 16 unsigned 4-bit limbs, every limb value
// 0..15 and every bit 0/1 is exact in e4m3, and each f32 accumulator sums at most L <= 2^20 terms
// of at most 15 < 2^24 / 2^20, so every partial sum is an exact integer; the limbs are recombined
// mod 2^64 after the loop.
//
// Operand tables (built once per layer, e-contiguous so that a 4-byte word covers 4 consecutive e):
//   BB1[j][e], BB2[j'][e] = e4m3(bit j of b1[e]) / e4m3(bit j' of b2[e])   (64 x Epad bytes each)
//   TL8[c][e_lo]           = e4m3(limb c % 16 of coefficient c / 16 of T_lo[e_lo]) (1024 x L)
// The A fragment of pair rows (j, j') is the BB2 tile of the 64 rows j' loaded with ldmatrix and
// ANDed with the BB1 bytes of the CTA's row j (0x38 & 0x38 = 0x38 = 1.0, anything & 0 = 0).
#include "kernels.h"

namespace mpc3 {

namespace {

constexpr int S_PAIRS = 128;       // pairs (rows) per CTA: two values of j x 64 values of j'
constexpr int S_COLS = 256;        // limb columns per CTA = 16 coefficients x 16 limbs
constexpr int S_KB = 128;          // e per pipeline stage
constexpr int S_ROWB = S_KB + 16;  // padded bytes per row of a staged tile

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldsm_x4(const void* p, unsigned& r0, unsigned& r1, unsigned& r2,
                                        unsigned& r3) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(s));
}

__device__ __forceinline__ void mma_e4m3(float c[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
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

// BB[j * Epad + e] = 0x38 if bit j of words[e] else 0 (for 16 consecutive e per thread).
__global__ void k_bit_bytes(const u64* __restrict__ words, long long Epad, unsigned char* __restrict__ BB) {
  const long long chunks = Epad / 16;
  const long long total = 64 * chunks;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
       w += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(w / chunks);
    const long long e0 = (w % chunks) * 16;
    unsigned v[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if ((words[e0 + i] >> j) & 1ull) v[i >> 2] |= 0x38u << (8 * (i & 3));
    uint4 out;
    out.x = v[0]; out.y = v[1]; out.z = v[2]; out.w = v[3];
    *reinterpret_cast<uint4*>(BB + (long long)j * Epad + e0) = out;
  }
}

// S_hi[e_hi][p][coeff] for pairs p = 64 j + j'.  Grid (32 pair tiles, 4 coefficient tiles, n_hi),
// 256 threads: warp (wm, wn) owns pairs wm*64 .. +63 of the tile (j = 2 blockIdx.x + wm, all j')
// and limb columns wn*64 .. +63 (4 coefficients).
__global__ void __launch_bounds__(256, 1)
k_trunc_s_mma(const unsigned char* __restrict__ BB1, const unsigned char* __restrict__ BB2,
              long long Epad, const unsigned char* __restrict__ TL8, long long L,
              u64* __restrict__ S_hi) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* Ls = smem;                               // [2][S_COLS][S_ROWB] limb tile
  unsigned char* Ps = Ls + 2 * S_COLS * S_ROWB;           // [2][64][S_ROWB]     b2 bytes, rows j'
  unsigned char* Qs = Ps + 2 * 64 * S_ROWB;               // [2][2][S_ROWB]      b1 bytes, rows j

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int pt = blockIdx.x;
  const int ct = blockIdx.y;
  const long long ehi = blockIdx.z;
  const int grp = lane >> 2, q = lane & 3;

  const unsigned char* Lsrc = TL8 + (long long)(ct * S_COLS) * L;
  const long long ebase = ehi * L;
  const int nkb = (int)(L / S_KB);

  auto issue = [&](int kb, int stage) {
    const long long e0 = (long long)kb * S_KB;
    unsigned char* ld = Ls + stage * S_COLS * S_ROWB;
#pragma unroll
    for (int it = 0; it < 8; ++it) {                 // 256 columns x 8 chunks of 16 bytes
      const int chunk = tid + it * 256;
      const int col = chunk >> 3, part = chunk & 7;
      cp_async16(ld + col * S_ROWB + part * 16, Lsrc + (long long)col * L + e0 + part * 16);
    }
    unsigned char* pd = Ps + stage * 64 * S_ROWB;
#pragma unroll
    for (int it = 0; it < 2; ++it) {                 // 64 rows j' x 8 chunks
      const int chunk = tid + it * 256;
      const int row = chunk >> 3, part = chunk & 7;
      cp_async16(pd + row * S_ROWB + part * 16, BB2 + (long long)row * Epad + ebase + e0 + part * 16);
    }
    if (tid < 16) {                                  // 2 rows j x 8 chunks
      const int row = tid >> 3, part = tid & 7;
      cp_async16(Qs + (stage * 2 + row) * S_ROWB + part * 16,
                 BB1 + (long long)(2 * pt + row) * Epad + ebase + e0 + part * 16);
    }
    cp_async_commit();
  };

  float acc[4][8][4];
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[t][u][i] = 0.f;

  // ldmatrix row addresses: lanes 0-7 rows 0-7 (bytes 0-15), 8-15 rows 8-15, 16-23 rows 0-7
  // (bytes 16-31), 24-31 rows 8-15 (bytes 16-31)
  const int lrow = (lane & 7) + ((lane >> 3) & 1) * 8;
  const int lcol = (lane >> 4) * 16;

  issue(0, 0);
  for (int kb = 0; kb < nkb; ++kb) {
    const int stage = kb & 1;
    cp_async_wait0();
    __syncthreads();
    if (kb + 1 < nkb) issue(kb + 1, stage ^ 1);
    const unsigned char* Lt = Ls + stage * S_COLS * S_ROWB;
    const unsigned char* Pt = Ps + stage * 64 * S_ROWB;
    const unsigned char* Qt = Qs + (stage * 2 + wm) * S_ROWB;
#pragma unroll 1
    for (int g = 0; g < 4; ++g) {                    // k32 steps of this stage
      const unsigned mlo = *reinterpret_cast<const unsigned*>(Qt + g * 32 + 4 * q);
      const unsigned mhi = *reinterpret_cast<const unsigned*>(Qt + g * 32 + 16 + 4 * q);
      unsigned a[4][4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        ldsm_x4(Pt + (16 * t + lrow) * S_ROWB + g * 32 + lcol, a[t][0], a[t][1], a[t][2], a[t][3]);
        a[t][0] &= mlo; a[t][1] &= mlo; a[t][2] &= mhi; a[t][3] &= mhi;
      }
#pragma unroll
      for (int u2 = 0; u2 < 4; ++u2) {               // two n8 tiles per ldmatrix.x4
        unsigned b00, b01, b10, b11;
        // rows: n = wn*64 + 16 u2 + (lane & 7) + 8 ((lane >> 4) & 1); bytes (lane >> 3 & 1) * 16
        const int nrow = wn * 64 + 16 * u2 + (lane & 7) + ((lane >> 4) & 1) * 8;
        const int ncol = ((lane >> 3) & 1) * 16;
        ldsm_x4(Lt + nrow * S_ROWB + g * 32 + ncol, b00, b01, b10, b11);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          mma_e4m3(acc[t][2 * u2], a[t][0], a[t][1], a[t][2], a[t][3], b00, b01);
          mma_e4m3(acc[t][2 * u2 + 1], a[t][0], a[t][1], a[t][2], a[t][3], b10, b11);
        }
      }
    }
  }

  // recombine limbs: coefficient v (0..3) of this warp = tiles u = 2v (limbs 0..7), 2v+1 (8..15)
#pragma unroll
  for (int t = 0; t < 4; ++t) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      u64 lo = 0, hi = 0;   // rows grp and grp + 8
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int u = 2 * v + h;
        const int l0 = 8 * h + 2 * q;
        lo += ((u64)__float2uint_rn(acc[t][u][0]) << (4 * l0)) +
              ((u64)__float2uint_rn(acc[t][u][1]) << (4 * (l0 + 1)));
        hi += ((u64)__float2uint_rn(acc[t][u][2]) << (4 * l0)) +
              ((u64)__float2uint_rn(acc[t][u][3]) << (4 * (l0 + 1)));
      }
      lo += __shfl_xor_sync(0xffffffffu, lo, 1);
      lo += __shfl_xor_sync(0xffffffffu, lo, 2);
      hi += __shfl_xor_sync(0xffffffffu, hi, 1);
      hi += __shfl_xor_sync(0xffffffffu, hi, 2);
      if (q == v) {
        const int pr = pt * S_PAIRS + wm * 64 + 16 * t + grp;
        const int coeff = ct * 16 + wn * 4 + v;
        S_hi[(ehi * 4096 + pr) * 64 + coeff] = lo;
        S_hi[(ehi * 4096 + pr + 8) * 64 + coeff] = hi;
      }
    }
  }
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

size_t trunc_s_smem_bytes() { return (size_t)(2 * S_COLS + 2 * 64 + 2 * 2) * S_ROWB; }

void launch_trunc_limb_table(cudaStream_t st, const u64* Tlo, long long L, unsigned char* TL8) {
  const long long total = 1024 * (L / 16);
  long long g = (total + 255) / 256;
  if (g > (1ll << 20)) g = 1ll << 20;
  k_limb_table<<<(unsigned)g, 256, 0, st>>>(Tlo, L, TL8);
}

void launch_trunc_bit_bytes(cudaStream_t st, const u64* words, long long Epad, unsigned char* BB) {
  const long long total = 64 * (Epad / 16);
  long long g = (total + 255) / 256;
  if (g > (1ll << 20)) g = 1ll << 20;
  k_bit_bytes<<<(unsigned)g, 256, 0, st>>>(words, Epad, BB);
}

void launch_trunc_s_mma(cudaStream_t st, const unsigned char* BB1, const unsigned char* BB2,
                        long long Epad, const unsigned char* TL8, long long L, long long nhi,
                        u64* S_hi) {
  const size_t smem = trunc_s_smem_bytes();
  cudaFuncSetAttribute(k_trunc_s_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(4096 / S_PAIRS, 64 / 16, (unsigned)nhi);
  k_trunc_s_mma<<<grid, 256, smem, st>>>(BB1, BB2, Epad, TL8, L, S_hi);
}

void launch_fold_reduce_strided(cudaStream_t st, const u64* P, long long ld, int npairs, u64* out) {
  k_fold_reduce_strided<<<npairs, 128, 0, st>>>(P, ld, out);
}

}  // namespace mpc3
