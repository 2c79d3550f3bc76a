// gemm_ozaki.cu -- FP64 GEMM emulated on the BF16 tensor cores (error-free splitting, Ozaki, Ogita, Oishi &
// Rump, "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 2012), for the compact-WY updates and sketch
// products of Algorithms 1 and 3 on a GPU whose FP64 units are ~1/1600 of its BF16 tensor throughput.
//
// Splitting: row r of op(A) (length K) is scaled by 2^-e_r, where max_k |a_rk| < 2^(e_r - 1), and written
// as S = 7 signed base-256 digits per entry:  a = 2^e_r sum_s d_s 2^-8(s+1) + rem,  |d_s| <= 128,
// |rem| <= 2^-57 2^e_r < 2^-55 max_k |a_rk| -- every digit an exact BF16 value and every step exact in FP64.
// Columns of op(B) likewise (exponents f_c).
// Products: a digit product is at most 2^14, so over 64 of K the diagonal sum
// S_d = sum_{i+j=d} sum_k d^A_i d^B_j (d + 1 pairs) is an integer of magnitude <= (d + 1) 2^20 < 2^23: the
// tcgen05 MMA's FP32 accumulation is exact.  S_0 .. S_3 (<= 2^22) convert to integers exactly by a
// magic-number add (x + 1.5 2^23 holds round(x) in its low mantissa bits), S_4 by a round-to-nearest
// conversion instruction.  The epilogue adds S_0 2^32 + S_1 2^24 + S_2 2^16 + S_3 2^8 + S_4 into one int64
// per output (exact; a split covers at most 65536 of K, so it stays below 2^63) and the remaining
// S_5 2^-8 + S_6 2^-16 into an FP32 fraction whose integer part moves into the int64 after every read (its
// rounding is below 2^-59 of the row/column scale per read).  The digit products of diagonals 7..12 are
// dropped (at most 2^-51.4 max|a_r.| max|b_.c| per k, ~2^-56 for random digits).  At the end
// C = alpha 2^(e_r + f_c - 48) (acc + frac) + beta C, the FP64 value packed with integer instructions.
//
// Kernel (576 threads, persistent over 128 x 32 output tiles x K splits): warp 0 lane 0 loads the 7 + 7
// digit tiles of each 32-wide K chunk with two 3-D TMA loads (64-byte swizzle, 3-stage ring); warp 1 lane 0
// issues, per 16-wide K step and A digit a, one MMA of A_a against the B digits 0..6-a laid back to back
// (N = (7-a) 32), accumulating two chunks (64 of K) into one of two TMEM buffers of 7 x 32 columns used
// alternately; warps 2..17 read a buffer (tcgen05.ld) while the MMAs fill the other.  All mbarrier waits
// are bounded (RRF_TIMEOUT, drain, free TMEM, exit).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "rrf_internal.cuh"

namespace rrf {
namespace {

constexpr int kS = 7;            // digits per value
constexpr int BM = 128, BN = 32;
constexpr int KC = 32;           // K per chunk / stage (64 bytes of BF16: 64-byte swizzle)
constexpr int kStages = 3;
constexpr int kHarvest = 2;      // chunks accumulated in TMEM per epilogue read (64 of K)
constexpr int kEpiWarps = 16;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kBufCols = 256;    // TMEM columns between the two accumulator buffers (7 x BN = 224 used)
constexpr int kGroupM = 8;       // tile raster: groups of 8 row tiles, column tiles fastest inside a group
constexpr int64_t kMaxSplitK = 65536;  // K of one split: keeps the int64 accumulator below 2^63
constexpr long long kWaitCycles = 4000000000LL;
constexpr uint32_t kTileA = BM * KC * 2;   // 8 KB per slice
constexpr uint32_t kTileB = BN * KC * 2;   // 2 KB per slice
constexpr uint32_t kStageBytes = kS * (kTileA + kTileB);
constexpr float kMagic = 12582912.0f;      // 1.5 * 2^23: x + kMagic holds round(x) in its low bits, |x| <= 2^22
constexpr int kMagicBits = 0x4B400000;

struct OzParams {
  int64_t M, N, Kp;     // Kp: padded K (multiple of KC)
  int64_t kchunk;       // K per split (multiple of KC, <= kMaxSplitK)
  int64_t units;        // tiles_m * tiles_n * splits
  int tiles_m, tiles_n, splits;
  const int* ea;        // M row exponents
  const int* eb;        // N column exponents
  double alpha, beta;
  double* C;            // splits == 1: C (ldc); else partials [split][N][M]
  int64_t ldc;
  int ct;               // write C^T: element (row, col) at C[col + row ldc]
  int* status;
  int amode;            // alpha: 1 -> +1, 2 -> -1, 0 -> any other value
  int bmode;            // beta != 0 (decided on the host: no FP64 comparison in the kernel)
  long long stall_cycles;  // failure injection only (0 normally): the MMA warp first waits this long on a
                           // barrier nothing arrives on, then aborts
};

// Work unit u -> (row tile, column tile, split).  Splits outermost; inside a split, groups of kGroupM row
// tiles with the column tile varying fastest, so the CTAs resident at one time share digit tiles in L2.
__device__ __forceinline__ void unit_coords(const OzParams& p, int64_t u, int64_t& m0, int64_t& n0, int& split) {
  const int64_t tiles = (int64_t)p.tiles_m * p.tiles_n;
  split = (int)(u / tiles);
  const int64_t t = u - (int64_t)split * tiles;
  const int64_t per_group = (int64_t)kGroupM * p.tiles_n;
  const int64_t first = (t / per_group) * kGroupM;
  const int64_t gm = min((int64_t)kGroupM, (int64_t)p.tiles_m - first);
  const int64_t r = t % per_group;
  m0 = (first + r % gm) * BM;
  n0 = (r / gm) * BN;
}

__device__ __forceinline__ int unit_chunks(const OzParams& p, int split, int64_t& k0) {
  k0 = (int64_t)split * p.kchunk;
  const int64_t k1 = min(p.Kp, k0 + p.kchunk);
  return k1 > k0 ? (int)((k1 - k0) / KC) : 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) { return mbar_wait_for(bar, parity, kWaitCycles); }
// All 7 digit slices of a tile in one load: box (32 of K, rows, 7 slices), slices stacked in shared memory.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
// K-major, 64-byte swizzle: 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw64(const void* p) {
  const uint64_t addr = (smem_u32(p) >> 4) & 0x3FFF;
  return addr | (uint64_t(512 >> 4) << 32) | (uint64_t(1) << 46) | (uint64_t(4) << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Exact integer value of a TMEM word holding an integer-valued FP32 x with |x| <= 2^22.
__device__ __forceinline__ int exact_int(uint32_t bits) {
  return __float_as_int(__fadd_rn(__uint_as_float(bits), kMagic)) - kMagicBits;
}

// Exact integer value of an integer-valued FP32 word with |x| < 2^24, with integer instructions only (a
// conversion instruction would run on the FP64 pipe): x = m 2^(e - 150) with the implicit bit in m.
__device__ __forceinline__ int exact_int_wide(uint32_t bits) {
  const int e = (int)((bits >> 23) & 0xFFu);  // 0 only for x = 0; 127..150 for 1 <= |x| < 2^24
  const int m = (int)((bits & 0x7FFFFFu) | 0x800000u);
  const int v = (e >= 127) ? (m >> (150 - e)) : 0;
  return (bits >> 31) ? -v : v;
}

// The rare exponents (subnormal or overflowing results) take the FP64 path, kept out of line so that the
// compiler does not predicate its FP64 instructions into every output.
__device__ __noinline__ double scaled_fp64(long long W, int x) { return ldexp((double)W, x); }
__device__ __noinline__ double times_alpha(double alpha, double v) { return alpha * v; }

// (acc + ta) 2^x as an FP64 value, for an exact integer acc and a fraction |ta| <= 1/2, with integer
// instructions only: this GPU's FP64 pipe does ~2 operations per clock per SM, far too few for a
// conversion, an add and a scaling per output.  The fixed-point value W = acc 2^10 + round(ta 2^10) (acc
// alone once |acc| >= 2^52, where the fraction is below the result's precision) is rounded to 53 bits,
// to nearest even, and packed with its exponent.  Subnormal or overflowing results take the FP64 path.
__device__ __forceinline__ double fixed_to_double(long long acc, float ta, int x) {
  const unsigned long long aa = acc < 0 ? 0ull - (unsigned long long)acc : (unsigned long long)acc;
  long long W = acc;
  int xs = x;
  if (aa < (1ull << 52)) {
    W = acc * 1024 + exact_int(__float_as_uint(ta * 1024.f));  // |ta 2^10| <= 2^9: exact rounding
    xs = x - 10;
  }
  if (W == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)W & 0x8000000000000000ull;
  const unsigned long long mag = W < 0 ? 0ull - (unsigned long long)W : (unsigned long long)W;
  const int lz = __clzll((long long)mag);
  const unsigned long long top = mag << lz;  // leading one at bit 63
  unsigned long long m = top >> 11;          // 53 significant bits
  const unsigned long long rem = top & 0x7FFull;
  m += (rem > 0x400ull || (rem == 0x400ull && (m & 1ull))) ? 1ull : 0ull;
  int e = 63 - lz + xs;                      // exponent of the leading bit
  if (m >> 53) {
    m >>= 1;
    ++e;
  }
  if (e < -1022 || e > 1023) return scaled_fp64(W, xs);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// Persistent kernel: each CTA walks work units blockIdx.x, blockIdx.x + gridDim.x, ...  The 32-wide K
// chunks of all its units form one stream g = 0, 1, ...: chunk g uses smem stage g % kStages and TMEM
// accumulator buffer g % 2, so the MMAs of chunk g + 1 run while the epilogue folds chunk g.
__global__ void __launch_bounds__(kThreads, 1)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                      const __grid_constant__ OzParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ __align__(8) uint64_t acc_full[2];
  __shared__ __align__(8) uint64_t acc_empty[2];
  __shared__ __align__(8) uint64_t never_bar;  // failure injection: nothing ever arrives on it
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    mbar_init(&never_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  int64_t issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      int64_t g = 0;
      bool run = true;
      for (int64_t u = blockIdx.x; u < p.units && run; u += gridDim.x) {
        int64_t m0, n0, k0;
        int split;
        unit_coords(p, u, m0, n0, split);
        const int nch = unit_chunks(p, split, k0);
        for (int i = 0; i < nch; ++i, ++g) {
          const int s = (int)(g % kStages);
          if (g >= kStages && !mbar_wait(&empty_bar[s], (uint32_t)((g / kStages) - 1) & 1)) {
            set_status(p.status, RRF_TIMEOUT);
            atomicExch(&abort_flag, 1);
            run = false;
            break;
          }
          if (*(volatile int*)&abort_flag) { run = false; break; }
          unsigned char* st = smem + s * kStageBytes;
          mbar_expect_tx(&full_bar[s], kStageBytes);
          const int kx = (int)(k0 + (int64_t)i * KC);
          tma_load_3d(st, &map_a, &full_bar[s], kx, (int)m0, 0);
          tma_load_3d(st + kS * kTileA, &map_b, &full_bar[s], kx, (int)n0, 0);
          issued = g + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // One MMA per A digit a per 16-wide K step: D[a .. 6] += A_a [B_0 .. B_{6-a}]^T.  The B digit tiles sit
      // back to back in shared memory, so they form one K-major operand of N = (7 - a) BN rows whose
      // products land on the diagonals a + j, stored contiguously in TMEM (diagonal d at column d BN).
      // Round h accumulates kHarvest chunks (64 of K) into TMEM buffer h % 2 before the epilogue reads it.
      const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BM >> 4) << 24);
      int64_t g = 0, h = 0;  // chunks consumed (shared-memory ring), rounds committed (TMEM ring)
      bool run = true;
      if (p.stall_cycles > 0 && !mbar_wait_for(&never_bar, 0, p.stall_cycles)) {
        set_status(p.status, RRF_TIMEOUT);
        atomicExch(&abort_flag, 1);
        run = false;
      }
      for (int64_t u = blockIdx.x; u < p.units && run; u += gridDim.x) {
        int64_t m0, n0, k0;
        int split;
        unit_coords(p, u, m0, n0, split);
        const int nch = unit_chunks(p, split, k0);
        for (int c0 = 0; c0 < nch && run; c0 += kHarvest) {
          const int bf = (int)(h & 1);
          if (h >= 2 && !mbar_wait(&acc_empty[bf], (uint32_t)((h >> 1) - 1) & 1)) {
            set_status(p.status, RRF_TIMEOUT);
            atomicExch(&abort_flag, 1);
            run = false;
            break;
          }
          const int c1 = min(nch, c0 + kHarvest);
          bool issued_any = false;
          for (int i = c0; i < c1; ++i, ++g) {
            const int s = (int)(g % kStages);
            if (!mbar_wait(&full_bar[s], (uint32_t)(g / kStages) & 1)) {
              set_status(p.status, RRF_TIMEOUT);
              atomicExch(&abort_flag, 1);
              run = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned char* st = smem + s * kStageBytes;
            const uint64_t db = smem_desc_sw64(st + kS * kTileA);
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
#pragma unroll
              for (int a = 0; a < kS; ++a) {
                const uint64_t da = smem_desc_sw64(st + a * kTileA);
                const uint32_t idesc = idesc0 | ((uint32_t)(((kS - a) * BN) >> 3) << 17);
                mma_bf16(tmem + (uint32_t)(bf * kBufCols + a * BN), da + 2 * kk, db + 2 * kk, idesc,
                         (i > c0 || a > 0 || kk > 0) ? 1u : 0u);
              }
            }
            mma_commit(&empty_bar[s]);
            issued_any = true;
          }
          // commit the round (also a partial one cut short by a timeout, so that the wait below covers
          // every MMA issued before TMEM is released)
          if (issued_any) {
            mma_commit(&acc_full[bf]);
            ++h;
          }
        }
      }
      // the last MMAs must finish before TMEM is released
      if (h > 0) mbar_wait(&acc_full[(h - 1) & 1], (uint32_t)((h - 1) >> 1) & 1);
    }
  } else {
    // Epilogue warps ew = 0..15: TMEM lane quadrant (warp % 4) = 32 tile rows, columns 8 (ew / 4) .. +7.
    const bool beta_nz = p.bmode != 0;
    const int ew = warp - 2;
    const int quad = warp & 3;
    const int col0 = (ew >> 2) * 8;
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)col0;
    int64_t h = 0;
    for (int64_t u = blockIdx.x; u < p.units; u += gridDim.x) {
      int64_t m0, n0, k0;
      int split;
      unit_coords(p, u, m0, n0, split);
      const int nch = unit_chunks(p, split, k0);
      // acc: sum over rounds of S_0 2^32 + S_1 2^24 + S_2 2^16 + S_3 2^8 + S_4 (exact); ta: the rest,
      // S_5 2^-8 + S_6 2^-16, in the same unit, with its integer part moved into acc after every round.
      long long acc[8];
      float ta[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) { acc[c] = 0; ta[c] = 0.f; }
      // The tile's column exponents and (beta != 0) C values are loaded before the first harvest, so their
      // latency runs under the unit's MMAs; nothing else in this kernel writes this tile's C.
      const int64_t row = m0 + quad * 32 + lane;
      const bool direct = p.splits == 1;
      int ec[8];
      double cin[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t col = n0 + col0 + c;
        ec[c] = col < p.N ? p.eb[col] : 0;
        cin[c] = 0.0;
        if (direct && beta_nz && row < p.M && col < p.N) cin[c] = p.ct ? p.C[col + row * p.ldc] : p.C[row + col * p.ldc];
      }
      bool ok = true;
      for (int c0 = 0; c0 < nch; c0 += kHarvest, ++h) {
        const int bf = (int)(h & 1);
        if (!mbar_wait(&acc_full[bf], (uint32_t)(h >> 1) & 1)) {
          set_status(p.status, RRF_TIMEOUT);
          atomicExch(&abort_flag, 1);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t v[kS][8];
#pragma unroll
        for (int d = 0; d < kS; ++d) tmem_ld8(trow + (uint32_t)(bf * kBufCols + d * BN), v[d]);
        tmem_wait_ld();
        // the buffer may be refilled as soon as every warp holds its values
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[bf]);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          // Over a round of 64 of K, |S_d| <= (d + 1) 64 2^14: S_0 .. S_3 are within 2^22 and convert exactly
          // by the magic-number add; S_4 (up to 5 2^20) from its bit pattern.
          const int hi = exact_int(v[0][c]) * 256 + exact_int(v[1][c]);   // |.| < 2^29
          const int mid = exact_int(v[2][c]) * 256 + exact_int(v[3][c]);  // |.| < 2^30
          const int d4 = exact_int_wide(v[4][c]);
          float t = fmaf(__uint_as_float(v[5][c]), 0.00390625f, ta[c]);
          t = fmaf(__uint_as_float(v[6][c]), 1.52587890625e-05f, t);
          const float r = __fadd_rn(t, kMagic);
          const int ti = __float_as_int(r) - kMagicBits;
          ta[c] = __fsub_rn(t, __fsub_rn(r, kMagic));
          acc[c] += (long long)hi * 16777216LL + (long long)mid * 256LL + (long long)(d4 + ti);
        }
      }
      if (!ok || *(volatile int*)&abort_flag) break;
      if (row >= p.M) continue;
      const int er = p.ea[row];
      const bool has_beta = beta_nz;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t col = n0 + col0 + c;
        if (col >= p.N) continue;
        // value = 2^(e_r + f_c) sum_d S_d 2^-8(d+2) = (acc + ta) 2^(e_r + f_c - 48), assembled with integer
        // instructions; alpha = +-1 is a sign change, other alpha one FP64 multiply, beta != 0 one FP64 FMA.
        double v = nch > 0 ? fixed_to_double(acc[c], ta[c], er + ec[c] - 48) : 0.0;
        if (direct) {
          double* cp = p.ct ? p.C + col + row * p.ldc : p.C + row + col * p.ldc;
          if (p.amode == 2) v = __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
          else if (p.amode == 0) v = times_alpha(p.alpha, v);
          if (has_beta) v = fma(p.beta, cin[c], v);
          *cp = v;
        } else {
          p.C[((int64_t)split * p.N + col) * p.M + row] = v;
        }
      }
    }
  }
  __syncthreads();
  if (abort_flag && warp == 0 && lane == 0)
    for (int64_t i = (issued > kStages ? issued - kStages : 0); i < issued; ++i)
      mbar_wait(&full_bar[i % kStages], (uint32_t)(i / kStages) & 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
}

// The splitting works on the bit patterns with integer instructions only (the FP64 pipe of this GPU is
// ~60x slower than its integer pipe).  |x| orders like the bit pattern with the sign cleared.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
// e with |x| < 2^(e - 1) for the largest magnitude m (bit pattern, nonzero): frexp exponent + 1.
__device__ __forceinline__ int scale_exponent(unsigned long long m) {
  if (m == 0) return 0;
  const int E = (int)(m >> 52);
  if (E != 0) return E - 1021;
  return (64 - __clzll((long long)m)) - 1074 + 1;  // subnormal: m * 2^-1074
}

// BF16 of an integer |d| <= 128 (exact: at most 8 significant bits) without a conversion instruction (those
// run on the FP64 pipe): the magic-number add gives the FP32 value, whose upper half is the BF16 pattern.
__device__ __forceinline__ __nv_bfloat16 small_int_bf16(int d) {
  const float f = __fsub_rn(__int_as_float(kMagicBits + d), kMagic);
  return __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
}

// Row maxima (as bit patterns with the sign cleared) of X(r, k) = X[r sr + k sk]; mx must be zeroed first.
// sr == 1 (a row strided in memory): 32 rows x a slice of K per block, combined with atomicMax; otherwise
// (each row contiguous) one warp per row.
__global__ void oz_rowmax_kernel(int64_t rows, int64_t K, const double* __restrict__ X, int64_t sr, int64_t sk,
                                 unsigned long long* __restrict__ mx) {
  if (sr == 1) {
    __shared__ unsigned long long red[8][32];
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int64_t r = (int64_t)blockIdx.x * 32 + tx;
    unsigned long long m = 0;
    if (r < rows)
      for (int64_t k = (int64_t)blockIdx.y * 8 + ty; k < K; k += (int64_t)gridDim.y * 8) m = max(m, abs_bits(X[r + k * sk]));
    red[ty][tx] = m;
    __syncthreads();
    if (ty == 0 && r < rows) {
      for (int j = 1; j < 8; ++j) m = max(m, red[j][tx]);
      if (m != 0) atomicMax(&mx[r], m);
    }
  } else {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)(blockDim.x * blockDim.y) + threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x * blockDim.y) >> 5;
    for (int64_t r = wid; r < rows; r += nw) {
      unsigned long long m = 0;
      for (int64_t k = lane; k < K; k += 32) m = max(m, abs_bits(X[r * sr + k]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = max(m, (unsigned long long)__shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) mx[r] = m;
    }
  }
}

// Digits: D[s][r][k] (row stride Kp, slice stride rows * Kp), zero for k >= K.  32 x 32 tiles.
// x 2^(56 - e_r) is rounded to an integer X (|X| < 2^55; what it drops is below 2^-57 2^e_r) and X is
// written in balanced base 256: X = sum_s d_s 2^(8 (6 - s)), |d_s| <= 128.
// Also writes the row exponents e_r (max_k |X(r, k)| < 2^(e_r - 1), 0 for an all-zero row) from the maxima.
__global__ void oz_split_kernel(int64_t rows, int64_t K, int64_t Kp, const double* __restrict__ X, int64_t sr,
                                int64_t sk, const unsigned long long* __restrict__ mx, int* __restrict__ e,
                                __nv_bfloat16* __restrict__ D) {
  __shared__ long long tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, kb = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int j = ty; j < 32; j += 8) {
    // read with the contiguous index on tx
    int64_t r, k;
    if (sr == 1) { r = r0 + tx; k = kb + j; } else { r = r0 + j; k = kb + tx; }
    const long long v = (r < rows && k < K) ? __double_as_longlong(X[r * sr + k * sk]) : 0ll;
    if (sr == 1) tile[tx][j] = v; else tile[j][tx] = v;  // tile[row][k]
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + j, k = kb + tx;
    if (r >= rows || k >= Kp) continue;
    const int er = scale_exponent(mx[r]);
    if (blockIdx.y == 0 && tx == 0) e[r] = er;
    const unsigned long long bits = (unsigned long long)tile[j][tx];
    const unsigned long long a = bits & 0x7FFFFFFFFFFFFFFFull;
    const int E = (int)(a >> 52);
    long long mant = (long long)(a & 0xFFFFFFFFFFFFFull);
    int sh;
    if (E != 0) {
      mant |= 1ll << 52;
      sh = E - 1075 + 56 - er;
    } else {
      sh = -1074 + 56 - er;
    }
    long long Xi;
    if (a == 0 || sh <= -64) Xi = 0;
    else if (sh >= 0) Xi = mant << min(sh, 62);  // |x| < 2^(e - 1) keeps Xi below 2^55
    else Xi = (mant + (1ll << (-sh - 1))) >> (-sh);
    if (bits >> 63) Xi = -Xi;
#pragma unroll
    for (int sl = 0; sl < kS - 1; ++sl) {
      const int sb = 8 * (kS - 1 - sl);
      const long long dg = (Xi + (1ll << (sb - 1))) >> sb;
      Xi -= dg << sb;
      D[((int64_t)sl * rows + r) * Kp + k] = small_int_bf16((int)dg);
    }
    D[((int64_t)(kS - 1) * rows + r) * Kp + k] = small_int_bf16((int)Xi);
  }
}

__global__ void oz_reduce_kernel(int64_t M, int64_t N, int splits, const double* __restrict__ part, double alpha,
                                 double beta, double* __restrict__ C, int64_t ldc, int ct) {
  const int64_t total = M * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += part[sp * total + idx];
    double* cp = ct ? C + (idx / M) + (idx % M) * ldc : C + (idx % M) + (idx / M) * ldc;
    double v = alpha * s;
    if (beta != 0.0) v = fma(beta, *cp, v);
    *cp = v;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn oz_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

// 3-D map over the digit slices D[s][r][k]: dims (Kp, rows, 7); a box is (32, box_rows, 7) and lands in
// shared memory as 7 stacked (box_rows x 32) tiles with the 64-byte swizzle.  Rows past `rows` read zeros.
bool oz_map(CUtensorMap* map, const void* base, int64_t rows, int64_t Kp, int box_rows) {
  EncodeTiledFn fn = oz_encode_fn();
  if (fn == nullptr || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || ((Kp * 2) & 15) != 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)kS};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(rows * Kp * 2)};
  cuuint32_t box[3] = {(cuuint32_t)KC, (cuuint32_t)box_rows, (cuuint32_t)kS};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t oz_smem() { return (size_t)kStages * kStageBytes + 1024; }

int oz_splits(int64_t M, int64_t N, int64_t Kp) {
  const int sms = dev_info().sms;
  const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  const int64_t chunks = Kp / KC;
  int s = (int)((Kp + kMaxSplitK - 1) / kMaxSplitK);
  while (tiles * s < sms && chunks / (s * 2) >= 8 && s < 64) s *= 2;
  return s;
}

}  // namespace

bool ozaki_eligible(const GemmDesc& d, bool force) {
  const int64_t lo = std::min(d.M, d.N), hi = std::max(d.M, d.N);
  return hi >= 128 && lo >= 64 && d.K >= 32 && (force || 2.0 * d.M * d.N * d.K >= 2.0e7);
}

size_t ozaki_bound(int64_t m, int64_t n, int64_t b) {
  const int64_t mx = std::max(m, n);
  return std::max({ozaki_scratch_bytes(mx, std::max<int64_t>(b, 64), mx), ozaki_scratch_bytes(mx, mx, b),
                   ozaki_scratch_bytes(m, n, n)}) + 4096;
}

cudaError_t gemm_run(const GemmEngine& eng, const GemmDesc* d, int count, cudaStream_t s) {
  GemmDesc rest[4];
  int nrest = 0;
  for (int i = 0; i < count; ++i) {
    if (d[i].M <= 0 || d[i].N <= 0) continue;
    if (eng.emulate && eng.oz != nullptr && ozaki_eligible(d[i], eng.force)) {
      GemmDesc e = d[i];
      bool ct = false;
      if (e.M < e.N) {  // C^T = op(B)^T op(A)^T: put the long side on M
        std::swap(e.M, e.N);
        std::swap(e.A, e.B);
        std::swap(e.lda, e.ldb);
        const int ta = e.ta;
        e.ta = !e.tb;
        e.tb = !ta;
        ct = true;
      }
      if (ozaki_scratch_bytes(e.M, e.N, e.K) <= eng.oz_bytes) {
        cudaError_t err = gemm_ozaki(e, ct, eng.oz, eng.oz_bytes, eng.status, s, eng.max_ctas);
        if (err != cudaSuccess) return err;
        continue;
      }
    }
    rest[nrest++] = d[i];
  }
  if (nrest == 0) return cudaSuccess;
  return gemm_f64(rest, nrest, eng.scratch, eng.scratch_bytes, s);
}

size_t ozaki_scratch_bytes(int64_t M, int64_t N, int64_t K) {
  const int64_t Kp = (K + KC - 1) / KC * KC;
  size_t b = align_up((size_t)kS * M * Kp * 2, 256) + align_up((size_t)kS * N * Kp * 2, 256);
  b += align_up(sizeof(int) * M, 256) + align_up(sizeof(int) * N, 256);
  b += align_up(sizeof(unsigned long long) * (M + N), 256);
  b += align_up((size_t)oz_splits(M, N, Kp) * M * N * sizeof(double), 256);
  return b;
}

cudaError_t gemm_ozaki(const GemmDesc& d, bool out_transposed, char* scratch, size_t scratch_bytes, int* status,
                       cudaStream_t s, int max_ctas) {
  if (d.M <= 0 || d.N <= 0) return cudaSuccess;
  const int64_t M = d.M, N = d.N, K = d.K;
  const int64_t Kp = (K + KC - 1) / KC * KC;
  if (ozaki_scratch_bytes(M, N, K) > scratch_bytes) return cudaErrorInvalidValue;
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = scratch + off; off += align_up(bytes, 256); return p; };
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(take((size_t)kS * M * Kp * 2));
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(take((size_t)kS * N * Kp * 2));
  int* ea = reinterpret_cast<int*>(take(sizeof(int) * M));
  int* eb = reinterpret_cast<int*>(take(sizeof(int) * N));
  unsigned long long* mxa = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * (M + N)));
  unsigned long long* mxb = mxa + M;
  const int splits = oz_splits(M, N, Kp);
  double* part = reinterpret_cast<double*>(take((size_t)splits * M * N * sizeof(double)));
  // op(A)(m, k) = A[m + k lda] or A[k + m lda]; op(B)^T(n, k) = op(B)(k, n) = B[k + n ldb] or B[n + k ldb]
  const int64_t asr = d.ta ? d.lda : 1, ask = d.ta ? 1 : d.lda;
  const int64_t bsr = d.tb ? 1 : d.ldb, bsk = d.tb ? d.ldb : 1;
  const int sms = dev_info().sms;
  cudaError_t e0 = cudaMemsetAsync(mxa, 0, sizeof(unsigned long long) * (M + N), s);
  if (e0 != cudaSuccess) return e0;
  const unsigned kslices = (unsigned)std::min<int64_t>(std::max<int64_t>((K + 255) / 256, 1), 64);
  auto rowmax = [&](int64_t rows, const double* X, int64_t sr, int64_t sk, unsigned long long* mx) {
    if (sr == 1)
      oz_rowmax_kernel<<<dim3((unsigned)((rows + 31) / 32), kslices), dim3(32, 8), 0, s>>>(rows, K, X, sr, sk, mx);
    else
      oz_rowmax_kernel<<<(unsigned)(sms * 8), dim3(32, 8), 0, s>>>(rows, K, X, sr, sk, mx);
    count_launch();
  };
  rowmax(M, d.A, asr, ask, mxa);
  rowmax(N, d.B, bsr, bsk, mxb);
  oz_split_kernel<<<dim3((unsigned)((M + 31) / 32), (unsigned)(Kp / 32)), dim3(32, 8), 0, s>>>(M, K, Kp, d.A, asr, ask,
                                                                                            mxa, ea, As);
  count_launch();
  oz_split_kernel<<<dim3((unsigned)((N + 31) / 32), (unsigned)(Kp / 32)), dim3(32, 8), 0, s>>>(N, K, Kp, d.B, bsr, bsk,
                                                                                            mxb, eb, Bs);
  count_launch();
  CUtensorMap ma, mb;
  if (!oz_map(&ma, As, M, Kp, BM) || !oz_map(&mb, Bs, N, Kp, BN)) return cudaErrorInvalidValue;
  static std::atomic<bool> attr{false};  // set once per process (one GPU each)
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(ozaki_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  OzParams p;
  p.M = M; p.N = N; p.Kp = Kp;
  p.kchunk = ((Kp / KC + splits - 1) / splits) * KC;
  p.tiles_m = (int)((M + BM - 1) / BM);
  p.tiles_n = (int)((N + BN - 1) / BN);
  p.splits = splits;
  p.units = (int64_t)p.tiles_m * p.tiles_n * splits;
  p.ea = ea; p.eb = eb;
  p.alpha = d.alpha; p.beta = d.beta;
  p.amode = d.alpha == 1.0 ? 1 : (d.alpha == -1.0 ? 2 : 0);
  p.bmode = d.beta != 0.0 ? 1 : 0;
  p.C = splits == 1 ? d.C : part;
  p.ldc = d.ldc;
  p.ct = out_transposed ? 1 : 0;
  p.status = status;
  const Inject inj = inject_state();
  p.stall_cycles = inj.kind == RRF_INJECT_GEMM_STALL ? inj.value : 0;
  const unsigned grid = (unsigned)std::min<int64_t>(p.units, max_ctas > 0 ? std::min(max_ctas, sms) : sms);
  // profiled work: the FP64 product's 2 M N K, and the tensor work 28 x 2 M N Kp of the digit products
  // algorithmic bytes: the 7 BF16 digit slices of op(A) and op(B) read once, C written once (read once more
  // when beta != 0; split partials instead when K is split)
  const double abytes = 14.0 * (double)(M + N) * Kp + 8.0 * M * N * (splits > 1 ? splits : (d.beta != 0.0 ? 2 : 1));
  cudaEvent_t ev_end = profile_launch_begin(1, 2.0 * M * N * K, 56.0 * M * N * Kp, s, abytes);
  ozaki_gemm_kernel<<<grid, kThreads, oz_smem(), s>>>(ma, mb, p);
  count_launch();
  if (ev_end != nullptr) cudaEventRecord(ev_end, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  const int64_t blocks = std::min<int64_t>((M * N + 255) / 256, (int64_t)sms * 16);
  oz_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(M, N, splits, part, d.alpha, d.beta, d.C, d.ldc, p.ct);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rrf

using namespace rrf;

extern "C" size_t rrf_gemm_emulated_workspace(int64_t m, int64_t n, int64_t k) {
  if (m < 1 || n < 1 || k < 1) return kHeaderBytes;
  return kHeaderBytes + ozaki_scratch_bytes(std::max(m, n), std::min(m, n), k) + 256;
}

extern "C" rrf_status rrf_gemm_emulated(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                                        const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                                        double* C, int64_t ldc, void* workspace, size_t ws_bytes, void* stream) {
  clear_arg_error();
  const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && transa != 'N' && transa != 'n') { set_arg_error(1); return RRF_INVALID_ARG; }
  if (!tb && transb != 'N' && transb != 'n') { set_arg_error(2); return RRF_INVALID_ARG; }
  if (std::max(m, n) < 128 || std::min(m, n) < 64) { set_arg_error(3); return RRF_UNSUPPORTED; }
  if (k < 32) { set_arg_error(5); return RRF_UNSUPPORTED; }
  if (A == nullptr || lda < std::max<int64_t>(1, ta ? k : m)) { set_arg_error(8); return RRF_INVALID_ARG; }
  if (B == nullptr || ldb < std::max<int64_t>(1, tb ? n : k)) { set_arg_error(10); return RRF_INVALID_ARG; }
  if (C == nullptr || ldc < std::max<int64_t>(1, m)) { set_arg_error(13); return RRF_INVALID_ARG; }
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) { set_arg_error(14); return RRF_INVALID_ARG; }
  if (ws_bytes < rrf_gemm_emulated_workspace(m, n, k)) { set_arg_error(15); return RRF_WORKSPACE_TOO_SMALL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  WsHeader* hdr = reinterpret_cast<WsHeader*>(workspace);
  RRF_CUDA_TRY(cudaMemsetAsync(hdr, 0, kHeaderBytes, s));
  GemmEngine eng;
  eng.oz = reinterpret_cast<char*>(workspace) + kHeaderBytes;
  eng.oz_bytes = ws_bytes - kHeaderBytes;
  eng.status = &hdr->status;
  eng.emulate = true;
  eng.force = true;
  GemmDesc g;
  g.M = m; g.N = n; g.K = k;
  g.A = A; g.lda = lda; g.ta = ta;
  g.B = B; g.ldb = ldb; g.tb = tb;
  g.C = C; g.ldc = ldc;
  g.alpha = alpha; g.beta = beta;
  RRF_CUDA_TRY(gemm_run(eng, &g, 1, s));
  return RRF_OK;
}
