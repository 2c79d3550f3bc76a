// panel_qr.cu -- Householder QR of a tall r x w panel (HQR of Sec. 2.4) and its compact-WY factor.
//
// The panel is spread by rows over NB co-resident CTAs (cooperative launch).  Column j needs two
// reductions over all rows -- sigma^2 = ||x(1:)||^2 of the column and the inner products with the
// remaining columns -- and the classic formulation would need a second one after the reflector is
// known (v^T P(:, k)).  Here the second is avoided: with v = (x - beta e1) / (alpha - beta),
//     v^T P(:, k) = (x^T P(:, k) - beta P(j, k)) / (alpha - beta),
// so one reduction of [sigma^2, x^T P(:, j+1:w)] plus the owner's copy of row j gives every CTA the
// reflector and all update coefficients.  One grid barrier per column.  Partial sums are combined in
// a fixed order (per slot: every 8th CTA per thread, then a fixed shuffle tree), so the result is
// bitwise deterministic.  Every barrier wait is bounded in time and records RRF_TIMEOUT in the
// workspace status word instead of hanging.
//
// The compact-WY factor (Schreiber & Van Loan) is built from the Gram matrix S = Y^T Y (through the
// caller's GEMM router when given) as the inverse of diag(1/tau) + striu(S), one column per warp.
#include <algorithm>

#include "rrf_internal.cuh"

namespace rrf {
namespace {

constexpr int NT = 256;
constexpr int kMaxW = 256;
constexpr long long kBarrierCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr int kMaxCtas = 160;                       // panel CTAs (one per SM at most)
constexpr int kTps = 8;                             // threads that share one slot of the partial-sum reduction

struct PanelArgs {
  int64_t r;
  int w;
  double* P;
  int64_t ldp;
  double* tau;
  double* Y;
  int64_t ldy;
  double* Rout;  // optional w x w copy of R (zeros below the diagonal)
  int64_t ldr;
  double* partials;  // [2][w][nb]: slot-major so a warp reads one slot of all CTAs coalesced
  double* rowbuf;    // [2][w]
  WsHeader* hdr;
  int nb;
  int64_t rows_per;
  int staged;        // 1: this CTA's rows live in shared memory for the whole kernel
  unsigned bar_extra;  // participants the barrier waits for beyond the grid (0; 1 under failure injection)
  long long wait_cycles;  // how long a barrier wait lasts before it gives up
};

// Bounded grid barrier over nblocks participants, each wait limited to wait_cycles.  Returns false (and
// records RRF_TIMEOUT) if the wait gave up.
// The arrival is an acquire-release at GPU scope (after the CTA barrier it covers the whole CTA's writes),
// the wait an acquire, so no full fence is needed on either side.
__device__ bool grid_sync(WsHeader* hdr, unsigned nblocks, long long wait_cycles, unsigned& gen, int* s_fail) {
  __syncthreads();
  if (threadIdx.x == 0) {
    *s_fail = 0;
    const unsigned target = gen + 1;
    unsigned arrived;
    // acq_rel: the last arrival also acquires every earlier arrival's writes (it reads them next)
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(&hdr->bar_count) : "memory");
    if (arrived == nblocks - 1) {
      atomicExch(&hdr->bar_count, 0u);  // ordered before the release below; read only after it
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&hdr->bar_gen), "r"(target) : "memory");
    } else {
      const long long t0 = clock64();
      unsigned g;
      for (;;) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(&hdr->bar_gen) : "memory");
        if (g == target) break;
        if (clock64() - t0 > wait_cycles) {
          set_status(&hdr->status, RRF_TIMEOUT);
          *s_fail = 1;
          break;
        }
      }
    }
    gen = target;
    if (*(volatile int*)&hdr->status == RRF_TIMEOUT) *s_fail = 1;
  }
  __syncthreads();
  return *s_fail == 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Partial sums of column j over this CTA's rows (local panel Pl, local row l = global row i0 + l):
// slot j = sum_{i>j} x_i^2, slot k>j = sum_{i>=j} x_i P(i,k).  Written to out[k * nb].
// Staged panels (odd column stride in shared memory): tps = NT / (w - j) threads per slot (a power of
// two) split the rows and combine by shuffles, so FP64 work is one FMA per element plus log2(tps) adds
// per slot -- on this GPU's narrow FP64 pipe a per-slot warp reduction would cost more than the dot
// product.  Unstaged panels (rows in global memory): a warp per slot, lanes over rows (coalesced).
__device__ void column_partials(const PanelArgs& a, int j, const double* Pl, int64_t ldl, int64_t i0, int64_t nloc,
                                double* xs, double* out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t l = tid; l < nloc; l += NT) xs[l] = (i0 + l >= j) ? Pl[l + (int64_t)j * ldl] : 0.0;
  __syncthreads();
  const int64_t lb = (j > i0) ? (j - i0) : 0;  // first local row with i >= j
  if (a.staged) {
    const int slots = a.w - j;
    int tps = 1;
    while (tps * 2 * slots <= NT && tps < 32) tps *= 2;
    const int k = j + tid / tps, sub = tid % tps;
    double acc = 0.0;
    if (k < a.w) {
      const double* pk = Pl + (int64_t)k * ldl;
      if (k == j) {
        for (int64_t l = lb + sub; l < nloc; l += tps)
          if (i0 + l > j) acc = fma(xs[l], xs[l], acc);
      } else {
        for (int64_t l = lb + sub; l < nloc; l += tps) acc = fma(xs[l], pk[l], acc);
      }
    }
    for (int o = tps / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (k < a.w && sub == 0) out[(int64_t)k * a.nb] = acc;
  } else {
    for (int k = j + warp; k < a.w; k += NT / 32) {
      double acc = 0.0;
      if (k == j) {
        for (int64_t l = lb + lane; l < nloc; l += 32)
          if (i0 + l > j) acc = fma(xs[l], xs[l], acc);
      } else {
        const double* pk = Pl + (int64_t)k * ldl;
        for (int64_t l = lb + lane; l < nloc; l += 32) acc = fma(xs[l], pk[l], acc);
      }
      acc = warp_sum(acc);
      if (lane == 0) out[(int64_t)k * a.nb] = acc;
    }
  }
  __syncthreads();
}

// Trailing update by reflector j (P(i, k) -= z_k v_i for i >= j, k > j; z pre-multiplied by tau) fused
// with the partial sums of column j + 1 (those of column_partials(j + 1)): column j + 1 is updated first
// and copied to xs, then one pass over the other columns updates each element and accumulates its product
// with xs -- one read of the local panel and one CTA barrier fewer than updating and summing apart.
__device__ void update_and_partials(const PanelArgs& a, int j, bool upd, double* Pl, int64_t ldl, int64_t i0,
                                    int64_t nloc, double* xs, const double* vs, const double* zk, double* out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j1 = j + 1;
  const int64_t lb = (j > i0) ? (j - i0) : 0;  // first local row with i >= j
  {
    double* p1 = Pl + (int64_t)j1 * ldl;
    const double z1 = zk[j1];
    for (int64_t l = tid; l < nloc; l += NT) {
      double x = p1[l];
      if (upd && l >= lb) {
        x = fma(-z1, vs[l], x);
        p1[l] = x;
      }
      xs[l] = (i0 + l >= j1) ? x : 0.0;
    }
  }
  __syncthreads();
  if (a.staged) {
    const int slots = a.w - j1;
    int tps = 1;
    while (tps * 2 * slots <= NT && tps < 32) tps *= 2;
    const int k = j1 + tid / tps, sub = tid % tps;
    double acc = 0.0;
    if (k < a.w) {
      if (k == j1) {
        for (int64_t l = lb + sub; l < nloc; l += tps)
          if (i0 + l > j1) acc = fma(xs[l], xs[l], acc);
      } else {
        double* pk = Pl + (int64_t)k * ldl;
        const double zz = zk[k];
        if (upd) {
          for (int64_t l = lb + sub; l < nloc; l += tps) {
            const double pv = fma(-zz, vs[l], pk[l]);
            pk[l] = pv;
            acc = fma(xs[l], pv, acc);
          }
        } else {
          for (int64_t l = lb + sub; l < nloc; l += tps) acc = fma(xs[l], pk[l], acc);
        }
      }
    }
    for (int o = tps / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (k < a.w && sub == 0) out[(int64_t)k * a.nb] = acc;
  } else {
    for (int k = j1 + warp; k < a.w; k += NT / 32) {
      double acc = 0.0;
      if (k == j1) {
        for (int64_t l = lb + lane; l < nloc; l += 32)
          if (i0 + l > j1) acc = fma(xs[l], xs[l], acc);
      } else {
        double* pk = Pl + (int64_t)k * ldl;
        const double zz = zk[k];
        for (int64_t l = lb + lane; l < nloc; l += 32) {
          double pv = pk[l];
          if (upd) {
            pv = fma(-zz, vs[l], pv);
            pk[l] = pv;
          }
          acc = fma(xs[l], pv, acc);
        }
      }
      acc = warp_sum(acc);
      if (lane == 0) out[(int64_t)k * a.nb] = acc;
    }
  }
  __syncthreads();
}

// Sum of the nb CTAs' partials of every slot k in [j, w) into red[k]: kTps threads per slot, each adding
// every kTps-th CTA's partial (L >= nb / kTps loads, all in flight before the first add), then a fixed
// shuffle tree -- deterministic, one L2 round trip per NT / kTps slots.  Every CTA computes all slots, so
// the adds on the FP64 pipe (nb + 2 kTps per slot) are sized exactly: no padding adds.
template <int L>
__device__ __forceinline__ void reduce_slots(const double* __restrict__ part, int nb, int j, int w, double* red) {
  const int tid = threadIdx.x;
  for (int kb = j; kb < w; kb += NT / kTps) {
    const int k = kb + tid / kTps, sub = tid % kTps;
    double sum = 0.0;
    if (k < w) {
      const double* pk = part + (int64_t)k * nb;
      double v[L];
#pragma unroll
      for (int t = 0; t < L; ++t) {
        const int c = sub + kTps * t;
        v[t] = c < nb ? __ldcg(pk + c) : 0.0;
      }
      sum = v[0];
#pragma unroll
      for (int t = 1; t < L; ++t)
        if (sub + kTps * t < nb) sum += v[t];
    }
#pragma unroll
    for (int o = 1; o < kTps; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (k < w && sub == 0) red[k] = sum;
  }
}

__global__ void __launch_bounds__(NT) panel_qr_kernel(const __grid_constant__ PanelArgs a) {
  extern __shared__ double smem[];
  __shared__ double red[kMaxW];
  __shared__ double zk[kMaxW];
  __shared__ double s_scalars[4];  // tau, beta, scal
  __shared__ int s_fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cta = blockIdx.x;
  const int64_t i0 = std::min<int64_t>((int64_t)cta * a.rows_per, a.r);
  const int64_t i1 = std::min<int64_t>(i0 + a.rows_per, a.r);
  const int64_t nloc = i1 - i0;
  const int w = a.w;
  double* xs = smem;                   // rows_per
  double* vs = smem + a.rows_per;      // rows_per
  double* Pl = a.P + i0;               // local panel: global rows, or staged copy
  int64_t ldl = a.ldp;
  if (a.staged) {
    Pl = smem + 2 * a.rows_per;
    ldl = a.rows_per | 1;  // odd stride: a thread per column reads distinct banks
    for (int k = warp; k < w; k += NT / 32)
      for (int64_t l = lane; l < nloc; l += 32) Pl[l + k * ldl] = a.P[(i0 + l) + (int64_t)k * a.ldp];
    __syncthreads();
  }
  unsigned gen = 0;
  if (tid == 0) gen = *(volatile unsigned*)&a.hdr->bar_gen;

  // Phase 0: partials of column 0.
  column_partials(a, 0, Pl, ldl, i0, nloc, xs, a.partials + cta);
  if (i0 == 0 && nloc > 0)
    for (int k = tid; k < w; k += NT) a.rowbuf[k] = Pl[(int64_t)k * ldl];
  if (!grid_sync(a.hdr, gridDim.x + a.bar_extra, a.wait_cycles, gen, &s_fail)) return;

  for (int j = 0; j < w; ++j) {
    const int par = j & 1;
    // Reduce the partial sums (the loads of P(j, k) above are in flight with them).
    const double* part = a.partials + (int64_t)par * w * a.nb;
    const double* row = a.rowbuf + (int64_t)par * w;
    for (int k = j + tid; k < w; k += NT) zk[k] = __ldcg(row + k);
    switch ((a.nb + 4 * kTps - 1) / (4 * kTps)) {  // loads per thread, rounded up to a multiple of 4
      case 1: reduce_slots<4>(part, a.nb, j, w, red); break;
      case 2: reduce_slots<8>(part, a.nb, j, w, red); break;
      case 3: reduce_slots<12>(part, a.nb, j, w, red); break;
      case 4: reduce_slots<16>(part, a.nb, j, w, red); break;
      case 5: reduce_slots<20>(part, a.nb, j, w, red); break;
      case 6: reduce_slots<24>(part, a.nb, j, w, red); break;
      case 7: reduce_slots<28>(part, a.nb, j, w, red); break;
      case 8: reduce_slots<32>(part, a.nb, j, w, red); break;
      case 9: reduce_slots<36>(part, a.nb, j, w, red); break;
      default: reduce_slots<40>(part, a.nb, j, w, red); break;
    }
    __syncthreads();
    if (tid == 0) {
      const double sig2 = red[j], alpha = zk[j];
      double tau = 0.0, beta = alpha, scal = 0.0;
      if (sig2 != 0.0) {
        const double nrm = sqrt(alpha * alpha + sig2);
        beta = (alpha >= 0.0) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      s_scalars[0] = tau;
      s_scalars[1] = beta;
      s_scalars[2] = scal;
      if (cta == 0) a.tau[j] = tau;
    }
    __syncthreads();
    const double tau = s_scalars[0], beta = s_scalars[1], scal = s_scalars[2];
    // z_k = v^T P(:, k) = (x^T P(:, k) - beta P(j, k)) / (alpha - beta); stored pre-multiplied by tau.
    for (int k = j + 1 + tid; k < w; k += NT) zk[k] = tau * ((red[k] - beta * zk[k]) * scal);
    // v over local rows (v_j = 1); column j becomes [beta; v(1:)].
    for (int64_t l = tid; l < nloc; l += NT) {
      const int64_t i = i0 + l;
      double v = 0.0;
      if (i == j) {
        v = 1.0;
        Pl[l + (int64_t)j * ldl] = beta;
      } else if (i > j) {
        v = (tau != 0.0) ? Pl[l + (int64_t)j * ldl] * scal : 0.0;
        Pl[l + (int64_t)j * ldl] = v;
      }
      vs[l] = v;
    }
    __syncthreads();
    if (j + 1 < w) {
      // Trailing update of the panel (P(i, k) -= tau z_k v_i for i >= j, k > j) with the partial sums of
      // column j + 1.
      update_and_partials(a, j, tau != 0.0, Pl, ldl, i0, nloc, xs, vs, zk,
                          a.partials + (int64_t)((j + 1) & 1) * w * a.nb + cta);
      if ((j + 1) >= i0 && (j + 1) < i1) {
        double* rb = a.rowbuf + (int64_t)((j + 1) & 1) * w;
        const int64_t lj = (j + 1) - i0;
        for (int k = j + 1 + tid; k < w; k += NT) rb[k] = Pl[lj + (int64_t)k * ldl];
      }
      if (!grid_sync(a.hdr, gridDim.x + a.bar_extra, a.wait_cycles, gen, &s_fail)) return;
    }
  }
  // Write back (staged), explicit reflectors Y (unit diagonal, zeros above), optional clean copy of R.
  for (int k = warp; k < w; k += NT / 32) {
    const double* pk = Pl + (int64_t)k * ldl;
    double* yk = a.Y + (int64_t)k * a.ldy;
    for (int64_t l = lane; l < nloc; l += 32) {
      const int64_t i = i0 + l;
      const double v = pk[l];
      if (a.staged) a.P[i + (int64_t)k * a.ldp] = v;
      yk[i] = (i < k) ? 0.0 : (i == k ? 1.0 : v);
      if (a.Rout != nullptr && i < w) a.Rout[i + (int64_t)k * a.ldr] = (i <= k) ? v : 0.0;
    }
  }
}

// Compact-WY factor from S = Y^T Y and tau (Puglisi; Joffrain, Low, Quintana-Orti, van de Geijn and Van Zee,
// "Accumulating Householder transformations, revisited", ACM TOMS 2006): with H_j = I - tau_j y_j y_j^T,
// H_0 ... H_{w-1} = I - Y Tf Y^T where Tf^{-1} = diag(1/tau) + striu(S).  Reflectors with tau_j = 0 are the
// identity and drop out: row and column j of Tf are zero, the rest is the inverse on the other indices.
// Columns of the inverse are independent -- Tf(j, j) = tau_j, Tf(i, j) = -tau_i sum_{i<l<=j} S(i, l) Tf(l, j)
// for i = j-1 .. 0 -- so each column is one warp's back substitution (lanes split the sum, fixed shuffle
// tree: deterministic), and the w columns run on w / 8 CTAs at once instead of w dependent steps on one.
// The rows of S a CTA's back substitutions read next are staged in shared memory kLarftRows at a time
// (coalesced, all loads in flight), so each step waits on shared memory, not on an L2 round trip.
constexpr int kLarftWarps = 8;
constexpr int kLarftRows = 12;
__global__ void __launch_bounds__(32 * kLarftWarps) larft_kernel(int w, const double* __restrict__ S, int64_t lds,
                                                                 const double* __restrict__ tau, double* Tf,
                                                                 int64_t ldt) {
  __shared__ double tcol[kLarftWarps][kMaxW];
  __shared__ double srow[kLarftRows][kMaxW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * kLarftWarps + warp;
  const int jmax = min(w, (blockIdx.x + 1) * kLarftWarps) - 1;  // last column of this CTA
  const bool active = j < w;
  double* t = tcol[warp];
  const double tj = active ? tau[j] : 0.0;
  if (active && lane == 0) t[j] = tj;
  __syncwarp();
  for (int ib = jmax; ib > 0; ib -= kLarftRows) {
    const int ilo = max(0, ib - kLarftRows);
    // srow[i - ilo][l] = S(l, i) = S(i, l) for ilo <= i < ib, i < l <= jmax
    const int span = jmax + 1;
    for (int idx = threadIdx.x; idx < (ib - ilo) * span; idx += 32 * kLarftWarps) {
      const int ii = idx / span, l = idx - ii * span, i = ilo + ii;
      if (l > i) srow[ii][l] = S[l + (int64_t)i * lds];
    }
    __syncthreads();
    if (active) {
      for (int i = min(ib, j) - 1; i >= ilo; --i) {
        const double ti = tau[i];
        double dot = 0.0;
        if (ti != 0.0 && tj != 0.0) {
          const double* si = srow[i - ilo];
          for (int l = i + 1 + lane; l <= j; l += 32) dot = fma(si[l], t[l], dot);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        }
        if (lane == 0) t[i] = (ti != 0.0 && tj != 0.0) ? -ti * dot : 0.0;
        __syncwarp();
      }
    }
    __syncthreads();
  }
  if (active)
    for (int i = lane; i < w; i += 32) Tf[i + (int64_t)j * ldt] = (i <= j) ? t[i] : 0.0;
}

// CTAs for an r-row panel.  Per column every CTA adds all nb partials of each slot (~nb FP64 adds) and
// updates its r / nb rows (2 r / nb FMAs) on a narrow FP64 pipe; nb ~ sqrt(2 r) balances the two.
int choose_nb(int64_t r) {
  const int sms = dev_info().sms;
  int64_t nb = 1;
  while (nb * nb < 2 * r) ++nb;
  return (int)std::max<int64_t>(1, std::min<int64_t>(nb, std::min(sms, kMaxCtas)));
}

}  // namespace

size_t panel_scratch_bytes(int64_t r, int64_t w) {
  const int nb = choose_nb(r);
  size_t bytes = align_up((size_t)2 * nb * w * sizeof(double), 256);  // partials
  bytes += align_up((size_t)2 * w * sizeof(double), 256);              // rowbuf
  bytes += align_up((size_t)w * w * sizeof(double), 256);              // Gram matrix
  GemmDesc g;
  g.M = w; g.N = w; g.K = r;
  bytes += gemm_scratch_bytes(&g, 1);
  return bytes;
}

cudaError_t panel_qr(int64_t r, int64_t w, double* P, int64_t ldp, double* tau, double* Y, int64_t ldy,
                     double* Tf, int64_t ldtf, double* Rout, int64_t ldr, double* scratch,
                     size_t scratch_bytes, WsHeader* hdr, cudaStream_t stream, const GemmEngine* eng) {
  if (w <= 0 || r <= 0) return cudaSuccess;
  if (w > kMaxW || r < w) return cudaErrorInvalidValue;
  int nb = choose_nb(r);
  if (eng != nullptr && eng->max_ctas > 0) nb = std::min(nb, eng->max_ctas);
  char* base = reinterpret_cast<char*>(scratch);
  size_t off = 0;
  double* partials = reinterpret_cast<double*>(base + off);
  off += align_up((size_t)2 * nb * w * sizeof(double), 256);
  double* rowbuf = reinterpret_cast<double*>(base + off);
  off += align_up((size_t)2 * w * sizeof(double), 256);
  double* gram = reinterpret_cast<double*>(base + off);
  off += align_up((size_t)w * w * sizeof(double), 256);
  if (off > scratch_bytes) return cudaErrorInvalidValue;

  // Reset the grid barrier counter (the generation word only ever advances).
  cudaError_t e = cudaMemsetAsync(&hdr->bar_count, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;

  PanelArgs a;
  a.r = r;
  a.w = (int)w;
  a.P = P;
  a.ldp = ldp;
  a.tau = tau;
  a.Y = Y;
  a.ldy = ldy;
  a.Rout = Rout;
  a.ldr = ldr;
  a.partials = partials;
  a.rowbuf = rowbuf;
  a.hdr = hdr;
  a.nb = nb;
  a.rows_per = (r + nb - 1) / nb;
  const Inject inj = inject_state();
  const bool stall = inj.kind == RRF_INJECT_PANEL_STALL;
  a.bar_extra = stall ? 1u : 0u;
  a.wait_cycles = stall ? inj.value : kBarrierCycles;
  constexpr size_t kSmemCap = 200 * 1024;
  size_t dyn = (size_t)2 * a.rows_per * sizeof(double);
  const size_t staged_bytes = dyn + (size_t)(a.rows_per | 1) * w * sizeof(double);
  a.staged = staged_bytes <= kSmemCap ? 1 : 0;
  if (a.staged) dyn = staged_bytes;
  // Function attributes belong to the device that is current when they are set: once per device (ids
  // 0..63; the entry point without a workspace may be called on any device of the process).
  static std::atomic<unsigned long long> attr_set{0};
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess || cur < 0 || cur >= 64) cur = 0;
  const unsigned long long bit = 1ull << cur;
  if (!(attr_set.load() & bit)) {
    e = cudaFuncSetAttribute(panel_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    if (e != cudaSuccess) return e;
    attr_set.fetch_or(bit);
  }
  if (dyn > kSmemCap) return cudaErrorInvalidValue;
  void* args[] = {(void*)&a};
  count_launch();
  // profiled work: HQR's 2 r w^2 - 2 w^3 / 3 flops; algorithmic bytes: the panel read and written and Y written
  cudaEvent_t ev_end = profile_launch_begin(3, 2.0 * r * w * w - 2.0 * w * w * w / 3.0, 0.0, stream,
                                            24.0 * (double)r * w);
  e = cudaLaunchCooperativeKernel((const void*)panel_qr_kernel, dim3(nb), dim3(NT), args, dyn, stream);
  if (ev_end != nullptr) cudaEventRecord(ev_end, stream);
  if (e != cudaSuccess) return e;
  if (Tf != nullptr) {
    GemmDesc g;
    g.M = w; g.N = w; g.K = r;
    g.A = Y; g.lda = ldy; g.ta = 1;
    g.B = Y; g.ldb = ldy; g.tb = 0;
    g.C = gram; g.ldc = w;
    g.alpha = 1.0;
    g.beta = 0.0;
    e = (eng != nullptr) ? gemm_run(*eng, &g, 1, stream)
                         : gemm_f64(&g, 1, reinterpret_cast<double*>(base + off), scratch_bytes - off, stream);
    if (e != cudaSuccess) return e;
    larft_kernel<<<(unsigned)((w + kLarftWarps - 1) / kLarftWarps), 32 * kLarftWarps, 0, stream>>>((int)w, gram, w, tau,
                                                                                                Tf, ldtf);
    count_launch();
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace rrf
