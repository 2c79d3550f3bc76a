// jacobi.cu -- one-sided (Hestenes) Jacobi SVD of the b x b core R(1:b, 1:b) of Algorithm 3 (and of
// the last block), on one thread-block cluster.
//
// FP64 on GB300 runs at ~2 DFMA/clk/SM, so a single SM would need ~10 ms for a 128 x 128 SVD; the
// cluster spreads the rows of M and of the accumulated V over CL CTAs (8, or 16 for c > 128 where the
// device schedules such clusters; distributed shared memory):
// each CTA computes its partial column norms / inner products for all pairs of one round, the
// partials are summed in rank order through DSMEM after one cluster barrier, every CTA derives the
// identical rotation, and applies it to its own rows.  Pairs follow the round-robin (tournament)
// ordering, so each round rotates c/2 disjoint pairs at once.  The rotation rule and stopping test
// are Hestenes': skip when |gamma| <= tol sqrt(alpha beta) (tol = c 2^-53), otherwise
// zeta = (beta - alpha)/(2 gamma), t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2)), cs = 1/sqrt(1+t^2),
// sn = cs t; stop after a sweep without rotations, or after one whose rotations all had
// |gamma| <= 2^-30 sqrt(alpha beta) and |t| <= 2^-24 (cap 40 sweeps -> RRF_NOT_CONVERGED).
// With scratch, an FP32 pre-pass (one CTA for c <= 128, the cluster kernel in FP32 above) gives the
// starting V, two FP64 Newton-Schulz steps make it orthogonal, and the FP64 sweeps run on M V.
// Outputs: sigma_k = ||m_k|| sorted descending (ties by index), u_k = m_k / sigma_k, and each pair
// signed so the largest-magnitude entry of v_k (first on ties) is positive.  A zero sigma_k leaves
// u_k for the Gram-Schmidt completion kernel.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "rrf_internal.cuh"

namespace cg = cooperative_groups;

namespace rrf {
namespace {

constexpr int NT = 256;
constexpr int kMaxC = 256;
constexpr int kMaxSweeps = 40;
// FP32 pre-pass: one CTA for c <= kPreMaxC, the cluster kernel in FP32 for larger c.
constexpr int kPreThreads = 1024;
constexpr int kPreMinC = 32;
constexpr int kPreMaxC = 128;
constexpr int kPreSweeps = 10;
constexpr int kPreLd = kPreMaxC;  // column stride (floats) of the one-CTA pre-pass

struct JacobiArgs {
  int c;
  int rp;  // rows per CTA
  const double* M;
  int64_t ldm;
  double* Us;
  int64_t ldu;
  double* s;
  double* Vs;
  int64_t ldv;
  const double* V0;  // optional starting V (c x c, orthogonal); null = identity
  int64_t ldv0;
  WsHeader* hdr;
  int max_sweeps;    // FP64 sweeps before RRF_NOT_CONVERGED (kMaxSweeps; lower only under failure injection)
};

__device__ __forceinline__ void round_pair(int t, int k, int ne, int& p, int& q) {
  // circle method over ne (even) players: player 0 fixed, players 1..ne-1 rotate.
  int a, b;
  if (k == 0) {
    a = 0;
    b = 1 + t % (ne - 1);
  } else {
    a = 1 + (t + k) % (ne - 1);
    b = 1 + (t - k + (ne - 1)) % (ne - 1);
  }
  p = min(a, b);
  q = max(a, b);
}

// CL: cluster size (16 where the GPU schedules such clusters, else 8), given again at launch.
// PRE: FP32 pre-pass for c > 128 -- sweeps on M 2^-e in FP32 (tolerance 2^-16, at most kPreSweeps) and
// only the accumulated V (as FP64) written to a.Vs; the FP64 sweeps then start from it.
template <int CL, bool PRE>
__global__ void __launch_bounds__(NT, 1) jacobi_kernel(const __grid_constant__ JacobiArgs a) {
  using T = typename std::conditional<PRE, float, double>::type;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int c = a.c, rp = a.rp, ldl = rp + 1;  // local column stride (padded)
  T* Ml = smem;                              // [c][ldl]
  T* Vl = smem + (size_t)c * ldl;            // [c][ldl]
  T* part = Vl + (size_t)c * ldl;            // [2][CL][kMaxC/2][3]: every CTA's partials, pushed
  double* nrm = reinterpret_cast<double*>(part + 2 * CL * (kMaxC / 2) * 3);  // [kMaxC] squared norms
  double* vmax = nrm + kMaxC;                     // [kMaxC] partial max |v|
  int* vidx = reinterpret_cast<int*>(vmax + kMaxC);  // [kMaxC] row of the max
  __shared__ int s_rot, s_big;
  __shared__ T s_cs[kMaxC / 2], s_sn[kMaxC / 2];
  __shared__ int s_rotf[kMaxC / 2];
  __shared__ double s_sig[kMaxC];
  __shared__ double s_sign[kMaxC];
  __shared__ int s_rank[kMaxC];

  const int tid = threadIdx.x;
  const int r0 = rank * rp;
  const int nloc = max(0, min(rp, c - r0));
  // The FP32 pre-pass scales M by 2^-e (max |M| < 2^e, the same e in every CTA: each reads all of M).
  int ex = 0;
  if (PRE) {
    __shared__ double s_mx[NT / 32];
    double mx = 0.0;
    for (int idx = tid; idx < c * c; idx += NT) mx = fmax(mx, fabs(a.M[(idx % c) + (int64_t)(idx / c) * a.ldm]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) s_mx[tid >> 5] = mx;
    __syncthreads();
    mx = 0.0;
    for (int w = 0; w < NT / 32; ++w) mx = fmax(mx, s_mx[w]);
    if (mx > 0.0) frexp(mx, &ex);
  }
  // Load my rows of M; V starts as V0 (or the identity).
  for (int idx = tid; idx < c * rp; idx += NT) {
    const int col = idx / rp, i = idx % rp;
    const int gi = r0 + i;
    const double mv = (i < nloc) ? a.M[gi + (int64_t)col * a.ldm] : 0.0;
    Ml[col * ldl + i] = PRE ? (T)ldexp(mv, -ex) : (T)mv;
    if (a.V0 != nullptr)
      Vl[col * ldl + i] = (i < nloc) ? (T)a.V0[gi + (int64_t)col * a.ldv0] : (T)0;
    else
      Vl[col * ldl + i] = (i < nloc && gi == col) ? (T)1 : (T)0;
  }
  if (tid == 0) {
    s_rot = 0;
    s_big = 0;
  }
  cluster.sync();

  const int ne = c + (c & 1);
  const int npairs = ne / 2;
  const int rounds = ne - 1;
  const double tol = (double)c * 0x1p-53;
  // threads per pair (power of two, <= 32)
  int tpp = 1;
  while (tpp * 2 * npairs <= NT && tpp < 32) tpp *= 2;
  const int grp = tid / tpp, sub = tid % tpp;
  const bool active = grp < npairs;
  int par = 0;
  int sweep = 0;
  bool converged = false;
  const int max_sweeps = PRE ? kPreSweeps : a.max_sweeps;
  for (sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    for (int t = 0; t < rounds; ++t) {
      int p = 0, q = 0;
      if (active) round_pair(t, grp, ne, p, q);
      const bool real = active && q < c;
      // (1) partial alpha, beta, gamma over my rows.
      T al = 0, be = 0, ga = 0;
      if (real) {
        const T* mp = Ml + p * ldl;
        const T* mq = Ml + q * ldl;
        for (int i = sub; i < nloc; i += tpp) {
          const T x = mp[i], y = mq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
      }
      for (int o = tpp / 2; o > 0; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
      }
      // (2) push my partials into every CTA's buffer (remote stores do not stall), one cluster
      // barrier, then sum the local copies in rank order: identical totals on every CTA.
      T* slot = part + ((size_t)(par * CL + rank) * (kMaxC / 2) + grp) * 3;
      if (active && sub == 0) {
#pragma unroll
        for (int rr = 0; rr < CL; ++rr) {
          T* dst = cluster.map_shared_rank(slot, rr);
          dst[0] = al;
          dst[1] = be;
          dst[2] = ga;
        }
      }
      cluster.sync();
      // (3) thread g < npairs sums pair g's partials in rank order and derives its rotation, so these FP64
      // sequences (division, square roots) run in npairs / 32 fully active warps rather than in every warp
      // with one active lane per pair: on this GPU's narrow FP64 pipe a warp instruction costs the same
      // whatever its active lanes.  Results go through shared memory to the lanes that rotate.
      if (tid < npairs) {
        int gp, gq;
        round_pair(t, tid, ne, gp, gq);
        T gcs = 1, gsn = 0;
        int grot = 0;
        if (gq < c) {
          T A = 0, B = 0, G = 0;
#pragma unroll
          for (int rr = 0; rr < CL; ++rr) {
            const T* rp3 = part + ((size_t)(par * CL + rr) * (kMaxC / 2) + tid) * 3;
            A += rp3[0];
            B += rp3[1];
            G += rp3[2];
          }
          if (PRE) {
            if (G != 0.f && G * G > 0x1p-32f * (A * B)) {  // tolerance 2^-16, squared
              const float zeta = __fdividef(B - A, 2.f * G);
              const float tt = __fdividef(copysignf(1.f, zeta), fabsf(zeta) + __fsqrt_rn(fmaf(zeta, zeta, 1.f)));
              gcs = rsqrtf(fmaf(tt, tt, 1.f));
              gsn = gcs * tt;
              grot = 1;
              s_rot = 1;
            }
          } else {
          const double sab = sqrt(A * B);
          if (G != 0.0 && fabs(G) > tol * sab) {
            const double zeta = (B - A) / (2.0 * G);
            const double tt = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            gcs = 1.0 / sqrt(1.0 + tt * tt);
            gsn = gcs * tt;
            grot = 1;
            s_rot = 1;
            if (fabs(G) > 0x1p-30 * sab || fabs(tt) > 0x1p-24) s_big = 1;
          }
          }
        }
        s_cs[tid] = gcs;
        s_sn[tid] = gsn;
        s_rotf[tid] = grot;
      }
      __syncthreads();
      const T cs = active ? s_cs[grp] : (T)1, sn = active ? s_sn[grp] : (T)0;
      const int rot = active ? s_rotf[grp] : 0;
      if (real && rot) {
        T* mp = Ml + p * ldl;
        T* mq = Ml + q * ldl;
        T* vp = Vl + p * ldl;
        T* vq = Vl + q * ldl;
        for (int i = sub; i < nloc; i += tpp) {
          const T x = mp[i], y = mq[i];
          mp[i] = cs * x - sn * y;
          mq[i] = sn * x + cs * y;
          const T u = vp[i], v = vq[i];
          vp[i] = cs * u - sn * v;
          vq[i] = sn * u + cs * v;
        }
      }
      par ^= 1;
      __syncthreads();
    }
    __syncthreads();
    // Converged after a sweep without rotations, or after one whose every rotation had both
    // |gamma| <= 2^-30 sqrt(alpha beta) and |t| <= 2^-24.  A rotation of (p, q) by sin s moves the
    // normalized inner product of p with any other column by about |s| |gamma_qr| sqrt(alpha_q / alpha_p),
    // which these two bounds keep below 2^-53.5 (for alpha_q >= 2 alpha_p, s sqrt(alpha_q/alpha_p) is
    // itself ~2 |gamma_pq| / sqrt(alpha_p alpha_q)); over the c - 1 rotations of a column that stays
    // below the tolerance c 2^-53, so the next sweep would rotate nothing that matters.  The bound on t
    // matters for clusters: a core close to a multiple of an orthogonal matrix has tiny gamma but
    // alpha ~ beta, hence rotations up to pi/4 that mix columns and leave them non-orthogonal at the
    // level of gamma itself.  Every CTA holds the same totals, so all take the same decision.
    converged = (s_rot == 0) || (!PRE && s_big == 0);
    __syncthreads();
    if (tid == 0) {
      s_rot = 0;
      s_big = 0;
    }
    __syncthreads();
  }
  if (PRE) {  // the pre-pass hands over V only
    if (rank == 0 && tid == 0) a.hdr->flags[2] = sweep;  // diagnostics
    for (int idx = tid; idx < c * nloc; idx += NT) {
      const int k = idx / nloc, i = idx % nloc;
      a.Vs[(r0 + i) + (int64_t)k * a.ldv] = (double)Vl[k * ldl + i];
    }
    cluster.sync();
    return;
  }
  if (!converged && rank == 0 && tid == 0) set_status(&a.hdr->status, RRF_NOT_CONVERGED);
  if (rank == 0 && tid == 0) a.hdr->flags[1] = sweep;  // diagnostics: sweeps of the last SVD

  // Column norms and the position of each v_k's largest-magnitude entry.
  for (int k = tid; k < c; k += NT) {
    double ss = 0.0, best = -1.0;
    int bi = 0;
    for (int i = 0; i < nloc; ++i) {
      const double x = Ml[k * ldl + i];
      ss = fma(x, x, ss);
      const double av = fabs(Vl[k * ldl + i]);
      if (av > best) {
        best = av;
        bi = r0 + i;
      }
    }
    nrm[k] = ss;
    vmax[k] = best;
    vidx[k] = bi;
  }
  cluster.sync();
  for (int k = tid; k < c; k += NT) {
    double ss = 0.0, best = -1.0;
    int bi = 0, owner = 0;
    for (int rr = 0; rr < CL; ++rr) {
      ss += cluster.map_shared_rank(nrm, rr)[k];
      const double bv = cluster.map_shared_rank(vmax, rr)[k];
      if (bv > best) {
        best = bv;
        bi = cluster.map_shared_rank(vidx, rr)[k];
        owner = rr;
      }
    }
    s_sig[k] = sqrt(ss);
    // sign of v_k at its largest-magnitude entry (read from the owner's rows)
    const int li = bi - owner * rp;
    const double vv = cluster.map_shared_rank(Vl, owner)[k * ldl + li];
    s_sign[k] = (vv < 0.0) ? -1.0 : 1.0;
  }
  __syncthreads();
  for (int k = tid; k < c; k += NT) {
    int rk = 0;
    const double sk = s_sig[k];
    for (int j = 0; j < c; ++j) {
      const double sj = s_sig[j];
      rk += (sj > sk || (sj == sk && j < k)) ? 1 : 0;
    }
    s_rank[k] = rk;
  }
  __syncthreads();
  for (int idx = tid; idx < c * nloc; idx += NT) {
    const int k = idx / nloc, i = idx % nloc;
    const int dst = s_rank[k];
    const double sg = s_sign[k], sig = s_sig[k];
    const int gi = r0 + i;
    a.Vs[gi + (int64_t)dst * a.ldv] = sg * Vl[k * ldl + i];
    a.Us[gi + (int64_t)dst * a.ldu] = (sig > 0.0) ? sg * (Ml[k * ldl + i] / sig) : 0.0;
  }
  if (rank == 0)
    for (int k = tid; k < c; k += NT) {
      a.s[s_rank[k]] = s_sig[k];
      if (s_sig[k] == 0.0) a.hdr->flags[0] = 1;
    }
  cluster.sync();  // keep shared memory alive until every CTA is done reading it
}

// FP32 pre-pass (c <= 128, one CTA): Hestenes sweeps on R 2^-e (scaled into FP32 range) in shared memory,
// one warp per column pair (each lane holds 4 consecutive rows as a float4; columns padded to 128 rows
// with zeros), until a sweep without rotations at tolerance 2^-16 or kPreSweeps sweeps (a looser tolerance
// costs FP64 sweeps when singular values cluster, a tighter one meets FP32 rounding).  Only the accumulated rotation
// V32 leaves the kernel: it is a preconditioner, orthonormalized in FP64 afterwards.

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

__global__ void __launch_bounds__(kPreThreads, 1)
    jacobi_f32_prepass_kernel(int c, const double* __restrict__ M, int64_t ldm, double* __restrict__ Vout,
                              int64_t ldvo, int* sweeps_out) {
  extern __shared__ __align__(16) float sm32[];
  float* Ms = sm32;                  // [c][kPreLd], column k at k * kPreLd, rows >= c zero
  float* Vs = sm32 + c * kPreLd;     // [c][kPreLd]
  __shared__ unsigned char s_pair[kPreMaxC - 1][kPreMaxC / 2][2];
  __shared__ double s_part[kPreThreads / 32];
  __shared__ int s_rot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ne = c + (c & 1), npairs = ne / 2, rounds = ne - 1;
  for (int idx = tid; idx < rounds * npairs; idx += kPreThreads) {
    int p, q;
    round_pair(idx / npairs, idx % npairs, ne, p, q);
    s_pair[idx / npairs][idx % npairs][0] = (unsigned char)p;
    s_pair[idx / npairs][idx % npairs][1] = (unsigned char)q;
  }
  double mx = 0.0;
  for (int idx = tid; idx < c * c; idx += kPreThreads) mx = fmax(mx, fabs(M[(idx % c) + (int64_t)(idx / c) * ldm]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_part[warp] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < kPreThreads / 32; ++w) mx = fmax(mx, s_part[w]);
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  for (int idx = tid; idx < c * kPreLd; idx += kPreThreads) {
    const int i = idx % kPreLd, k = idx / kPreLd;
    Ms[idx] = (i < c) ? (float)ldexp(M[i + (int64_t)k * ldm], -ex) : 0.f;
    Vs[idx] = (i == k) ? 1.f : 0.f;
  }
  if (tid == 0) s_rot = 0;
  __syncthreads();
  const float tol2 = 0x1p-32f;  // tolerance 2^-16, squared
  const int r4 = 4 * lane;
  int sweep = 0;
  for (; sweep < kPreSweeps; ++sweep) {
    for (int t = 0; t < rounds; ++t) {
      for (int g = warp; g < npairs; g += kPreThreads / 32) {
        const int p = s_pair[t][g][0], q = s_pair[t][g][1];
        if (q >= c) continue;
        float* mp = Ms + p * kPreLd + r4;
        float* mq = Ms + q * kPreLd + r4;
        const float4 x = ld4(mp), y = ld4(mq);
        float al = x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
        float be = y.x * y.x + y.y * y.y + y.z * y.z + y.w * y.w;
        float ga = x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        // approximate division / square roots suffice here: the FP64 sweeps decide the result
        if (ga != 0.f && ga * ga > tol2 * (al * be)) {
          const float zeta = __fdividef(be - al, 2.f * ga);
          const float tt = __fdividef(copysignf(1.f, zeta), fabsf(zeta) + __fsqrt_rn(fmaf(zeta, zeta, 1.f)));
          const float cs = rsqrtf(fmaf(tt, tt, 1.f));
          const float sn = cs * tt;
          st4(mp, make_float4(cs * x.x - sn * y.x, cs * x.y - sn * y.y, cs * x.z - sn * y.z, cs * x.w - sn * y.w));
          st4(mq, make_float4(sn * x.x + cs * y.x, sn * x.y + cs * y.y, sn * x.z + cs * y.z, sn * x.w + cs * y.w));
          float* vp = Vs + p * kPreLd + r4;
          float* vq = Vs + q * kPreLd + r4;
          const float4 u = ld4(vp), v = ld4(vq);
          st4(vp, make_float4(cs * u.x - sn * v.x, cs * u.y - sn * v.y, cs * u.z - sn * v.z, cs * u.w - sn * v.w));
          st4(vq, make_float4(sn * u.x + cs * v.x, sn * u.y + cs * v.y, sn * u.z + cs * v.z, sn * u.w + cs * v.w));
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    const bool done = (s_rot == 0);
    __syncthreads();
    if (done) break;
    if (tid == 0) s_rot = 0;
    __syncthreads();
  }
  if (tid == 0 && sweeps_out != nullptr) *sweeps_out = sweep;  // diagnostics
  for (int idx = tid; idx < c * c; idx += kPreThreads)
    Vout[(idx % c) + (int64_t)(idx / c) * ldvo] = (double)Vs[(idx % c) + (idx / c) * kPreLd];
}

// Gram-Schmidt completion of u_k for exactly-zero singular values (two passes against the columns
// already present, candidates e_0, e_1, ... in order).  Runs only when the Jacobi kernel flagged it.
__global__ void __launch_bounds__(NT) complete_kernel(int c, double* Us, int64_t ldu, const double* s,
                                                      WsHeader* hdr) {
  if (*(volatile int*)&hdr->flags[0] == 0) return;
  __shared__ double w[kMaxC];
  __shared__ double red[NT / 32];
  __shared__ double s_d;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < c; ++k) {
    if (s[k] > 0.0) continue;
    for (int e = 0; e < c; ++e) {
      for (int i = tid; i < c; i += NT) w[i] = (i == e) ? 1.0 : 0.0;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int j = 0; j < c; ++j) {
          if (j == k || (j > k && s[j] == 0.0)) continue;
          double d = 0.0;
          for (int i = tid; i < c; i += NT) d = fma(Us[i + (int64_t)j * ldu], w[i], d);
          for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
          if (lane == 0) red[warp] = d;
          __syncthreads();
          if (tid == 0) {
            double t = 0.0;
            for (int x = 0; x < NT / 32; ++x) t += red[x];
            s_d = t;
          }
          __syncthreads();
          const double dd = s_d;
          for (int i = tid; i < c; i += NT) w[i] -= dd * Us[i + (int64_t)j * ldu];
          __syncthreads();
        }
      }
      double nn = 0.0;
      for (int i = tid; i < c; i += NT) nn = fma(w[i], w[i], nn);
      for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
      if (lane == 0) red[warp] = nn;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int x = 0; x < NT / 32; ++x) t += red[x];
        s_d = sqrt(t);
      }
      __syncthreads();
      const double norm = s_d;
      if (norm > 0.5) {
        for (int i = tid; i < c; i += NT) Us[i + (int64_t)k * ldu] = w[i] / norm;
        __syncthreads();
        break;
      }
      __syncthreads();
    }
  }
  if (tid == 0) hdr->flags[0] = 0;
}

size_t jacobi_smem(int c, int cl, bool pre) {
  const int rp = (c + cl - 1) / cl;
  const size_t elem = pre ? sizeof(float) : sizeof(double);
  size_t b = ((size_t)2 * c * (rp + 1) + (size_t)2 * cl * (kMaxC / 2) * 3) * elem;
  b = (b + 15) / 16 * 16;
  return b + 2 * kMaxC * sizeof(double) + kMaxC * sizeof(int);
}

template <int CL, bool PRE>
cudaError_t set_jacobi_attrs() {
  if (CL > 8) {
    cudaError_t e = cudaFuncSetAttribute(jacobi_kernel<CL, PRE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(jacobi_kernel<CL, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)jacobi_smem(kMaxC, CL, PRE));
}

// 16-CTA clusters are not portable: use them when the device accepts the attribute and can schedule one.
int jacobi_cluster_size() {
  static int cl = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    cl = 8;
    if (set_jacobi_attrs<16, false>() != cudaSuccess || set_jacobi_attrs<16, true>() != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = jacobi_smem(kMaxC, 16, false);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, jacobi_kernel<16, false>, &cfg) == cudaSuccess && n > 0) cl = 16;
    cudaGetLastError();
  });
  return cl;
}

template <int CL, bool PRE>
cudaError_t launch_jacobi(const JacobiArgs& a, int c, cudaStream_t stream) {
  static std::atomic<bool> attr{false};  // set once per process (one GPU each)
  if (!attr) {
    cudaError_t e = set_jacobi_attrs<CL, PRE>();
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = jacobi_smem(c, CL, PRE);
  cfg.stream = stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, jacobi_kernel<CL, PRE>, a);
}

}  // namespace

size_t jacobi_scratch_bytes(int64_t c) {
  if (c < kPreMinC || c > kMaxC) return 0;
  GemmDesc g;
  g.M = c; g.N = c; g.K = c;
  return align_up((size_t)3 * c * c * sizeof(double), 256) + gemm_scratch_bytes(&g, 1);
}

cudaError_t jacobi_svd(int64_t c, const double* M, int64_t ldm, double* Us, int64_t ldu, double* s,
                       double* Vs, int64_t ldv, WsHeader* hdr, cudaStream_t stream, double* scratch,
                       size_t scratch_bytes) {
  if (c <= 0) return cudaSuccess;
  if (c > kMaxC) return cudaErrorInvalidValue;
  JacobiArgs a;
  a.c = (int)c;
  // 16 CTAs only pay off when each holds enough rows (c > 128); measured on GB300.  For c <= 128 an
  // 8-CTA cluster beats 2 or 4 CTAs even beside the trailing-update GEMMs (8192^2 randUTV, b = 128:
  // 675 ms with 8, 697 ms with 4, 781 ms with 2).
  const int cl = (c > 128) ? jacobi_cluster_size() : 8;
  a.rp = (int)((c + cl - 1) / cl);
  a.M = M;
  a.ldm = ldm;
  a.Us = Us;
  a.ldu = ldu;
  a.s = s;
  a.Vs = Vs;
  a.ldv = ldv;
  a.V0 = nullptr;
  a.ldv0 = 0;
  a.hdr = hdr;
  const Inject inj = inject_state();
  a.max_sweeps = inj.kind == RRF_INJECT_JACOBI_CAP ? (int)std::min<long long>(inj.value, kMaxSweeps) : kMaxSweeps;
  cudaError_t e;
  const size_t need = jacobi_scratch_bytes(c);
  if (scratch != nullptr && need > 0 && scratch_bytes >= need) {
    // Mixed precision: FP32 sweeps give V32; two Newton-Schulz steps X <- X + X (I - X^T X) / 2 make it
    // orthogonal to FP64 accuracy (the error squares each step); the FP64 sweeps then start from
    // M V0, whose columns are already nearly orthogonal, with V accumulated onto V0.
    double* X = scratch;
    double* Y = scratch + c * c;
    double* E = scratch + 2 * c * c;
    double* gs = reinterpret_cast<double*>(reinterpret_cast<char*>(scratch) +
                                           align_up((size_t)3 * c * c * sizeof(double), 256));
    const size_t gs_bytes = scratch_bytes - align_up((size_t)3 * c * c * sizeof(double), 256);
    static std::atomic<bool> attr_pre{false};  // set once per process (one GPU each)
    if (!attr_pre) {
      e = cudaFuncSetAttribute(jacobi_f32_prepass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(2 * kPreMaxC * kPreLd * sizeof(float)));
      if (e != cudaSuccess) return e;
      attr_pre = true;
    }
    if (c <= kPreMaxC) {
      jacobi_f32_prepass_kernel<<<1, kPreThreads, 2 * c * kPreLd * sizeof(float), stream>>>((int)c, M, ldm, X, c,
                                                                                      &hdr->flags[2]);
      e = cudaGetLastError();
    } else {
      JacobiArgs pa = a;
      pa.Vs = X;
      pa.ldv = c;
      pa.V0 = nullptr;
      e = (cl == 16) ? launch_jacobi<16, true>(pa, (int)c, stream) : launch_jacobi<8, true>(pa, (int)c, stream);  // c > 128
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    count_launch();
    if (e != cudaSuccess) return e;
    for (int it = 0; it < 2; ++it) {
      if ((e = fill_identity(c, c, E, c, stream)) != cudaSuccess) return e;
      GemmDesc g1;  // E = I - X^T X
      g1.M = c; g1.N = c; g1.K = c;
      g1.A = X; g1.lda = c; g1.ta = 1;
      g1.B = X; g1.ldb = c; g1.tb = 0;
      g1.C = E; g1.ldc = c;
      g1.alpha = -1.0; g1.beta = 1.0;
      if ((e = gemm_f64(&g1, 1, gs, gs_bytes, stream)) != cudaSuccess) return e;
      if ((e = copy_matrix(c, c, X, c, Y, c, stream)) != cudaSuccess) return e;
      GemmDesc g2 = g1;  // Y = X + X E / 2
      g2.A = X; g2.ta = 0;
      g2.B = E; g2.tb = 0;
      g2.C = Y;
      g2.alpha = 0.5; g2.beta = 1.0;
      if ((e = gemm_f64(&g2, 1, gs, gs_bytes, stream)) != cudaSuccess) return e;
      std::swap(X, Y);
    }
    GemmDesc g3;  // Y = M V0
    g3.M = c; g3.N = c; g3.K = c;
    g3.A = M; g3.lda = ldm; g3.ta = 0;
    g3.B = X; g3.ldb = c; g3.tb = 0;
    g3.C = Y; g3.ldc = c;
    g3.alpha = 1.0; g3.beta = 0.0;
    if ((e = gemm_f64(&g3, 1, gs, gs_bytes, stream)) != cudaSuccess) return e;
    a.M = Y;
    a.ldm = c;
    a.V0 = X;
    a.ldv0 = c;
  }
  e = cudaMemsetAsync(&hdr->flags[0], 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  switch (cl) {
    case 16: e = launch_jacobi<16, false>(a, (int)c, stream); break;
    default: e = launch_jacobi<8, false>(a, (int)c, stream); break;
  }
  count_launch();
  if (e != cudaSuccess) return e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  complete_kernel<<<1, NT, 0, stream>>>((int)c, Us, ldu, s, hdr);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rrf
