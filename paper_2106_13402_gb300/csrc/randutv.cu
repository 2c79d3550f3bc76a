// randutv.cu -- host driver of randUTV_basic (Algorithm 3) on one GPU.
//
// Per step i (offset o = b(i-1), trailing block T22 = T(o:, o:) of r x c):
//   G = randn(r, b); Y = T22^T G; q times { Z = T22 Y; Y = T22^T Z }      (sketch, optionally
//                                                                        re-orthonormalized)
//   panel HQR of Y -> (Yv, Tv);  [T(:, o:); V(:, o:)] <- [..](I - Yv Tv Yv^T)   (compact WY)
//   panel HQR of T(o:, o:o+b) -> (Yu, Tu, R);  T(o:, o+b:) <- (I - Yu Tu^T Yu^T) T(o:, o+b:),
//                                              U(:, o:) <- U(:, o:)(I - Yu Tu Yu^T)
//   Jacobi SVD of R -> (Us, D, Vs); U(:, I2) Us, V(:, J2) Vs, Us^T T(I2, J3), T(I1, J2) Vs,
//   T(I2 u I3, J2) = [D; 0].
// The last step (J3 empty) takes the SVD of the r x c remainder, through HQR first when r > c.
// Every product goes through the GEMM router (tensor-core FP64 emulation for large products by
// default); the BF16 sketch and the learned per-step q are options.  Everything is enqueued on the
// caller's stream and nothing is allocated; the learned policy synchronizes once per step.
#include <algorithm>
#include <cmath>
#include <vector>

#include "rrf_internal.cuh"

namespace rrf {

namespace {

struct RWs {
  WsHeader* hdr = nullptr;
  double *G = nullptr, *Y = nullptr, *Z = nullptr, *Yv = nullptr, *Yu = nullptr;
  double *Xa = nullptr, *Xb = nullptr, *Xc = nullptr, *Xd = nullptr;
  double *Wa = nullptr, *Wb = nullptr;
  double *tauv = nullptr, *tauu = nullptr, *Tv = nullptr, *Tu = nullptr, *Rs = nullptr;
  double *Us = nullptr, *Vs = nullptr, *sig = nullptr, *Qt = nullptr;
  double* panel = nullptr;
  size_t panel_bytes = 0;
  double* gemm = nullptr;
  size_t gemm_bytes = 0;
  GemmEngine eng;
  // BF16 sketch: T22 in BF16 twice (as stored, and transposed), the b-column operand, FP32 partials.
  __nv_bfloat16 *Tb = nullptr, *Tbt = nullptr, *Xh = nullptr;
  int64_t ldtb = 0, ldtbt = 0, ldxh = 0;
  float* part = nullptr;
  size_t part_bytes = 0;
  // learned q policy: features of the current step, the chosen q
  float* feat = nullptr;
  int* qdev = nullptr;
  // randUTV_boosted (oversampling p > 0): the k = b + p column sample, its SVD (Q_Y reflectors, R, U_R,
  // V_R, D), the left singular vectors W_Y, the recycled directions W_next, thin-Q scratch.
  double *Qk = nullptr, *Xk = nullptr, *Wy = nullptr, *Wn = nullptr, *Yq = nullptr, *tauq = nullptr;
  double *Tq = nullptr, *Ry = nullptr, *Uy = nullptr, *Vy = nullptr, *sy = nullptr, *S1 = nullptr, *S2 = nullptr;
  // early termination: e_i^2 of the Frobenius recurrence (steps + 1) and the reduction's partial sums
  double *e2 = nullptr, *fpart = nullptr;
  // b x b SVD beside the next step (see rrf_randutv): a second R / U_small / V_small / D set (the first is
  // Rs / Us / Vs / sig, used by even steps), the side stream's own header and SVD scratch
  double *Rs1 = nullptr, *Us1 = nullptr, *Vs1 = nullptr, *sig1 = nullptr;
  double* Wkk = nullptr;  // b x b scratch of the explicit thin Q (never R, which the side stream may read)
  WsHeader* hdr2 = nullptr;
  double* jscr = nullptr;
  size_t jscr_bytes = 0;
};

int64_t pad64(int64_t x) { return (x + 63) / 64 * 64; }

size_t layout(int64_t m, int64_t n, int64_t b, int64_t p, bool bf16, int gemm_mode, Arena& ar, RWs& w) {
  const int64_t mx = std::max(m, n);
  const int64_t kb = b + p;  // sample width (b for randUTV_basic)
  w.hdr = reinterpret_cast<WsHeader*>(ar.take<char>(kHeaderBytes));
  w.G = ar.take<double>(m * kb);
  w.Y = ar.take<double>(n * kb);
  w.Z = ar.take<double>(m * kb);
  w.Yv = ar.take<double>(n * b);
  w.Yu = ar.take<double>(m * b);
  w.Xa = ar.take<double>(mx * b);
  w.Xb = ar.take<double>(mx * b);
  w.Xc = ar.take<double>(mx * b);
  w.Xd = ar.take<double>(mx * b);
  w.Wa = ar.take<double>(b * mx);
  w.Wb = ar.take<double>(b * mx);
  w.Qt = ar.take<double>(mx * b);
  w.tauv = ar.take<double>(b);
  w.tauu = ar.take<double>(b);
  w.Tv = ar.take<double>(b * b);
  w.Tu = ar.take<double>(b * b);
  w.Rs = ar.take<double>(b * b);
  w.Us = ar.take<double>(b * b);
  w.Vs = ar.take<double>(b * b);
  w.sig = ar.take<double>(b);
  w.feat = ar.take<float>(16);
  w.qdev = ar.take<int>(4);
  w.e2 = ar.take<double>(std::min((m + b - 1) / b, (n + b - 1) / b) + 1);
  w.fpart = reinterpret_cast<double*>(ar.take<char>(frob_scratch_bytes()));
  w.Rs1 = ar.take<double>(b * b);
  w.Us1 = ar.take<double>(b * b);
  w.Vs1 = ar.take<double>(b * b);
  w.sig1 = ar.take<double>(b);
  w.Wkk = ar.take<double>(b * b);
  w.hdr2 = reinterpret_cast<WsHeader*>(ar.take<char>(kHeaderBytes));
  w.jscr_bytes = jacobi_scratch_bytes(std::min(b, n));
  w.jscr = reinterpret_cast<double*>(ar.take<char>(std::max<size_t>(w.jscr_bytes, 256)));
  if (p > 0) {
    w.Qk = ar.take<double>(m * kb);
    w.Xk = ar.take<double>(m * b);
    w.Wy = ar.take<double>(n * kb);
    w.Wn = ar.take<double>(n * p);
    w.Yq = ar.take<double>(mx * kb);
    w.tauq = ar.take<double>(kb);
    w.Tq = ar.take<double>(kb * kb);
    w.Ry = ar.take<double>(kb * kb);
    w.Uy = ar.take<double>(kb * kb);
    w.Vy = ar.take<double>(kb * kb);
    w.sy = ar.take<double>(kb);
    w.S1 = ar.take<double>(kb * kb);
    w.S2 = ar.take<double>(kb * kb);
  }
  w.panel_bytes = panel_scratch_bytes(mx, kb);
  w.panel = reinterpret_cast<double*>(ar.take<char>(w.panel_bytes));
  // split-K partials of the DFMA GEMMs; between them it also serves as the small SVD's scratch
  const int64_t steps = std::min((m + b - 1) / b, (n + b - 1) / b);
  const int64_t c_last = std::min(b, n - (steps - 1) * b);
  w.gemm_bytes = std::max({(size_t)16 * mx * kb * sizeof(double), jacobi_scratch_bytes(std::min(b, n)),
                           jacobi_scratch_bytes(c_last), p > 0 ? jacobi_scratch_bytes(std::min(kb, n)) : 0});
  w.gemm = reinterpret_cast<double*>(ar.take<char>(w.gemm_bytes));
  w.eng.scratch = w.gemm;
  w.eng.scratch_bytes = w.gemm_bytes;
  w.eng.status = w.hdr ? &w.hdr->status : nullptr;
  w.eng.emulate = gemm_mode != RRF_GEMM_NATIVE;
  w.eng.force = gemm_mode == RRF_GEMM_EMULATED;
  if (w.eng.emulate) {
    w.eng.oz_bytes = ozaki_bound(m, n, kb);
    w.eng.oz = ar.take<char>(w.eng.oz_bytes);
  }
  if (bf16) {
    w.ldtb = pad64(m);
    w.ldtbt = pad64(n);
    w.ldxh = pad64(mx);
    w.Tb = ar.take<__nv_bfloat16>(w.ldtb * n);
    w.Tbt = ar.take<__nv_bfloat16>(w.ldtbt * m);
    w.Xh = ar.take<__nv_bfloat16>(w.ldxh * b);
    w.part_bytes = (size_t)16 * mx * b * sizeof(float);
    w.part = ar.take<float>((size_t)16 * mx * b);
  }
  return ar.off;
}

GemmDesc gd(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, int ta, const double* B,
            int64_t ldb, int tb, double* C, int64_t ldc, double alpha = 1.0, double beta = 0.0) {
  GemmDesc g;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.ta = ta;
  g.B = B; g.ldb = ldb; g.tb = tb;
  g.C = C; g.ldc = ldc;
  g.alpha = alpha; g.beta = beta;
  return g;
}

// Thin explicit Q (rows x k) of a panel factored by panel_qr: Q = [I; 0] - Yr (Tr Yr(0:k,:)^T).
cudaError_t explicit_q(int64_t rows, int64_t k, const double* Yr, const double* Tr, double* Wkk, double* Q,
                       const RWs& w, cudaStream_t s) {
  GemmDesc g1 = gd(k, k, k, Tr, k, 0, Yr, rows, 1, Wkk, k);
  cudaError_t e = gemm_run(w.eng, &g1, 1, s);
  if (e != cudaSuccess) return e;
  e = fill_identity(rows, k, Q, rows, s);
  if (e != cudaSuccess) return e;
  GemmDesc g2 = gd(rows, k, k, Yr, rows, 0, Wkk, k, 0, Q, rows, -1.0, 1.0);
  return gemm_run(w.eng, &g2, 1, s);
}

// Y0 = T22^T G into Y: FP64 DFMA GEMM, or BF16 tensor cores after rounding T22 (both orientations) and G.
cudaError_t sketch_begin(int64_t r, int64_t c, int64_t b, const double* T22, int64_t ldt, bool bf16, const RWs& w,
                         cudaStream_t s) {
  if (!bf16) {
    GemmDesc g = gd(c, b, r, T22, ldt, 1, w.G, r, 0, w.Y, c);
    return gemm_run(w.eng, &g, 1, s);
  }
  cudaError_t e = to_bf16(r, c, T22, ldt, w.Tb, w.ldtb, s);                 // column j = T22(:, j)
  if (e == cudaSuccess) e = to_bf16_t(r, c, T22, ldt, w.Tbt, w.ldtbt, s);   // column i = T22(i, :)
  if (e == cudaSuccess) e = to_bf16(r, b, w.G, r, w.Xh, w.ldxh, s);
  if (e == cudaSuccess)
    e = gemm_bf16_tn(c, b, r, w.Tb, w.ldtb, w.Xh, w.ldxh, 1.0, w.Y, c, w.part, w.part_bytes, &w.hdr->status, s);
  return e;
}

// out = T22 * in (r x b) or T22^T * in (c x b), FP64 or BF16 (in is FP64; rounded for the BF16 form).
cudaError_t apply_t22(bool transposed, int64_t r, int64_t c, int64_t b, const double* T22, int64_t ldt, bool bf16,
                      const double* in, double* out, const RWs& w, cudaStream_t s) {
  const int64_t K = transposed ? r : c, M = transposed ? c : r;
  if (!bf16) {
    GemmDesc g = gd(M, b, K, T22, ldt, transposed ? 1 : 0, in, K, 0, out, M);
    return gemm_run(w.eng, &g, 1, s);
  }
  cudaError_t e = to_bf16(K, b, in, K, w.Xh, w.ldxh, s);
  if (e != cudaSuccess) return e;
  return gemm_bf16_tn(M, b, K, transposed ? w.Tb : w.Tbt, transposed ? w.ldtb : w.ldtbt, w.Xh, w.ldxh, 1.0, out, M,
                      w.part, w.part_bytes, &w.hdr->status, s);
}

// Orthonormal basis (explicit thin Q, rows x b) of X via the panel Householder QR; X is overwritten.
cudaError_t orthonormalize(int64_t rows, int64_t b, double* X, double* Qout, const RWs& w, cudaStream_t s) {
  cudaError_t e = panel_qr(rows, b, X, rows, w.tauu, w.Yu, rows, w.Tu, b, nullptr, 0, w.panel, w.panel_bytes, w.hdr, s, &w.eng);
  if (e == cudaSuccess) e = explicit_q(rows, b, w.Yu, w.Tu, w.Wkk, Qout, w, s);
  return e;
}

// q further applications: Y <- T22^T (T22 Y).  With reorth (always for BF16) the sample is orthonormalized
// before every application of T22 and of T22^T (Sec. 2.5 (ii)); `start` (optional) is an orthonormal
// basis of the current Y that the caller already has.  BF16 keeps only 8 bits: unorthonormalized,
// (T22^T T22)^q would lose everything below eps_bf16^(1/(2q+1)) sigma_max.
cudaError_t sketch_continue(int64_t r, int64_t c, int64_t b, const double* T22, int64_t ldt, int q, bool bf16,
                            bool reorth, const double* start, const RWs& w, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < q && e == cudaSuccess; ++j) {
    const double* yin = w.Y;
    if (reorth) {
      if (j == 0 && start != nullptr) {
        yin = start;
      } else {
        e = orthonormalize(c, b, w.Y, w.Qt, w, s);
        yin = w.Qt;
      }
    }
    if (e == cudaSuccess) e = apply_t22(false, r, c, b, T22, ldt, bf16, yin, w.Z, w, s);
    const double* zin = w.Z;
    if (reorth && e == cudaSuccess) {
      e = orthonormalize(r, b, w.Z, w.Qt, w, s);
      zin = w.Qt;
    }
    if (e == cudaSuccess) e = apply_t22(true, r, c, b, T22, ldt, bf16, zin, w.Y, w, s);
  }
  return e;
}

// ---- randUTV_boosted (Algorithm 2, Secs. 4.2-4.3) ----------------------------------------------------

// Explicit thin Q (rows x cols, ld ldq) of the columns of X (rows x cols, ld ldx, overwritten by the panel
// factorization), cols <= b + p: Q = [I; 0] - Yq (Tq Yq(0:cols, :)^T).
cudaError_t thin_q(int64_t rows, int64_t cols, double* X, int64_t ldx, double* Q, int64_t ldq, const RWs& w,
                   cudaStream_t s) {
  cudaError_t e = panel_qr(rows, cols, X, ldx, w.tauq, w.Yq, rows, w.Tq, cols, nullptr, 0, w.panel, w.panel_bytes,
                           w.hdr, s, &w.eng);
  GemmDesc g1 = gd(cols, cols, cols, w.Tq, cols, 0, w.Yq, rows, 1, w.S1, cols);
  if (e == cudaSuccess) e = gemm_run(w.eng, &g1, 1, s);
  if (e == cudaSuccess) e = fill_identity(rows, cols, Q, ldq, s);
  GemmDesc g2 = gd(rows, cols, cols, w.Yq, rows, 0, w.S1, cols, 0, Q, ldq, -1.0, 1.0);
  if (e == cudaSuccess) e = gemm_run(w.eng, &g2, 1, s);
  return e;
}

// The c x k sample of step i (k = b + pk) into w.Y.  Without recycled directions (step 1):
// G = randn(r, k), Y = (T22^T T22)^q T22^T G.  With them (every later step, W_next in w.Wn, ld c):
// G = randn(r, b), Y1 = (T22^T T22)^(q-1) T22^T G, X = T22 Y1, Z = orth(T22 W_next), X <- X - Z (Z^T X),
// Q = orth(X), Y = T22^T [Q, Z]: T22^T acts last on fresh and recycled directions alike.
cudaError_t boosted_sample(int64_t i, int64_t r, int64_t c, int64_t b, int64_t pk, bool recycle, int q,
                           const double* T22, int64_t ldt, uint64_t seed, const RWs& w, cudaStream_t s) {
  const int64_t k = b + pk;
  cudaError_t e;
  if (!recycle) {
    e = randn_f64(r, k, w.G, r, seed, (uint32_t)i, 1u, s);
    if (e == cudaSuccess) e = apply_t22(true, r, c, k, T22, ldt, false, w.G, w.Y, w, s);
    if (e == cudaSuccess) e = sketch_continue(r, c, k, T22, ldt, q, false, false, nullptr, w, s);
    return e;
  }
  double* Zq = w.Qk + b * r;  // orth(T22 W_next): the last pk columns of [Q, Z]
  e = randn_f64(r, b, w.G, r, seed, (uint32_t)i, 1u, s);
  if (e == cudaSuccess) e = apply_t22(true, r, c, b, T22, ldt, false, w.G, w.Y, w, s);
  if (e == cudaSuccess) e = sketch_continue(r, c, b, T22, ldt, q - 1, false, false, nullptr, w, s);
  if (e == cudaSuccess) e = apply_t22(false, r, c, b, T22, ldt, false, w.Y, w.Xk, w, s);
  if (e == cudaSuccess) e = apply_t22(false, r, c, pk, T22, ldt, false, w.Wn, w.Z, w, s);
  if (e == cudaSuccess) e = thin_q(r, pk, w.Z, r, Zq, r, w, s);
  GemmDesc g1 = gd(pk, b, r, Zq, r, 1, w.Xk, r, 0, w.S2, pk);
  if (e == cudaSuccess) e = gemm_run(w.eng, &g1, 1, s);
  GemmDesc g2 = gd(r, b, pk, Zq, r, 0, w.S2, pk, 0, w.Xk, r, -1.0, 1.0);
  if (e == cudaSuccess) e = gemm_run(w.eng, &g2, 1, s);
  if (e == cudaSuccess) e = thin_q(r, b, w.Xk, r, w.Qk, r, w, s);
  if (e == cudaSuccess) e = apply_t22(true, r, c, k, T22, ldt, false, w.Qk, w.Y, w, s);
  return e;
}

// Left singular vectors W_Y (c x k) of the sample in w.Y: Householder QR Y = Q_Y [R; 0], Jacobi SVD
// R = U_R D V_R^T, W_Y = Q_Y [U_R; 0] = [U_R; 0] - Yq (Tq (Yq(0:k, :)^T U_R)).  Leaves W_Y(:, 0:b) in w.Y,
// the panel that HQR_full factors into V_i.
cudaError_t boosted_svd(int64_t c, int64_t b, int64_t k, const RWs& w, cudaStream_t s) {
  cudaError_t e = panel_qr(c, k, w.Y, c, w.tauq, w.Yq, c, w.Tq, k, w.Ry, k, w.panel, w.panel_bytes, w.hdr, s,
                           &w.eng);
  if (e == cudaSuccess) e = jacobi_svd(k, w.Ry, k, w.Uy, k, w.sy, w.Vy, k, w.hdr, s, w.gemm, w.gemm_bytes);
  if (e == cudaSuccess) e = zero_matrix(c, k, w.Wy, c, s);
  if (e == cudaSuccess) e = copy_matrix(k, k, w.Uy, k, w.Wy, c, s);
  GemmDesc g1 = gd(k, k, k, w.Yq, c, 1, w.Uy, k, 0, w.S1, k);
  if (e == cudaSuccess) e = gemm_run(w.eng, &g1, 1, s);
  GemmDesc g2 = gd(k, k, k, w.Tq, k, 0, w.S1, k, 0, w.S2, k);
  if (e == cudaSuccess) e = gemm_run(w.eng, &g2, 1, s);
  GemmDesc g3 = gd(c, k, k, w.Yq, c, 0, w.S2, k, 0, w.Wy, c, -1.0, 1.0);
  if (e == cudaSuccess) e = gemm_run(w.eng, &g3, 1, s);
  if (e == cudaSuccess) e = copy_matrix(c, b, w.Wy, c, w.Y, c, s);
  return e;
}

// W_next = rows b.. of V_i^T W_Y(:, b:k), V_i^T = I - Yv Tv^T Yv^T: the recycled directions, expressed in
// the columns of the next trailing block (c - b rows, ld c - b, in w.Wn).
cudaError_t boosted_next(int64_t c, int64_t b, int64_t pk, const RWs& w, cudaStream_t s) {
  double* Wr = w.Wy + b * c;
  GemmDesc g1 = gd(b, pk, c, w.Yv, c, 1, Wr, c, 0, w.S1, b);
  cudaError_t e = gemm_run(w.eng, &g1, 1, s);
  GemmDesc g2 = gd(b, pk, b, w.Tv, b, 1, w.S1, b, 0, w.S2, b);
  if (e == cudaSuccess) e = gemm_run(w.eng, &g2, 1, s);
  GemmDesc g3 = gd(c, pk, b, w.Yv, c, 0, w.S2, b, 0, Wr, c, -1.0, 1.0);
  if (e == cudaSuccess) e = gemm_run(w.eng, &g3, 1, s);
  if (e == cudaSuccess) e = copy_matrix(c - b, pk, Wr + b, c, w.Wn, c - b, s);
  return e;
}

// A second stream (per host thread and device, created once) on which the b x b SVD of step i runs while
// the main stream applies U_i and samples step i + 1; events hand R over and the SVD back.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t ev_r[2] = {nullptr, nullptr}, ev_j[2] = {nullptr, nullptr};
  int dev = -1;
  bool ok = false;
};

SideStream* side_stream() {
  thread_local SideStream ss;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if (ss.ok && ss.dev == dev) return &ss;
  if (ss.dev != -1) return nullptr;  // created for another device: no side stream on this one
  ss.dev = dev;
  if (cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  for (int k = 0; k < 2; ++k)
    if (cudaEventCreateWithFlags(&ss.ev_r[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ss.ev_j[k], cudaEventDisableTiming) != cudaSuccess)
      return nullptr;
  ss.ok = true;
  return &ss;
}

// SMs the main stream leaves free while an SVD runs beside it: the 8-CTA cluster (its one-CTA FP32
// pre-pass runs first, on one of the same SMs).
constexpr int kSideReserve = 8;

rrf_status check_args(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q, double* U,
                      int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv, const rrf_opts* opts) {
  clear_arg_error();
  if (m < 1) { set_arg_error(1); return RRF_INVALID_ARG; }
  if (n < 1) { set_arg_error(2); return RRF_INVALID_ARG; }
  if (A == nullptr) { set_arg_error(3); return RRF_INVALID_ARG; }
  if (lda < m) { set_arg_error(4); return RRF_INVALID_ARG; }
  if (b < 1 || b > 256) { set_arg_error(5); return RRF_INVALID_ARG; }
  if (q < 0 || q > 16) { set_arg_error(6); return RRF_INVALID_ARG; }
  if (U == nullptr) { set_arg_error(7); return RRF_INVALID_ARG; }
  if (ldu < m) { set_arg_error(8); return RRF_INVALID_ARG; }
  if (T == nullptr) { set_arg_error(9); return RRF_INVALID_ARG; }
  if (ldt < m || (T == A && ldt != lda)) { set_arg_error(10); return RRF_INVALID_ARG; }
  if (V == nullptr) { set_arg_error(11); return RRF_INVALID_ARG; }
  if (ldv < n) { set_arg_error(12); return RRF_INVALID_ARG; }
  if (opts != nullptr) {
    if (opts->sketch_prec != RRF_SKETCH_FP64 && opts->sketch_prec != RRF_SKETCH_BF16) {
      set_arg_error(16); return RRF_INVALID_ARG;
    }
    if (opts->q_policy != RRF_Q_FIXED && opts->q_policy != RRF_Q_LEARNED) { set_arg_error(16); return RRF_INVALID_ARG; }
    if (opts->q_policy == RRF_Q_LEARNED && opts->q_per_block != nullptr) { set_arg_error(16); return RRF_INVALID_ARG; }
    if (opts->reserved[0] != 0) { set_arg_error(16); return RRF_INVALID_ARG; }
    const int64_t steps = std::min((m + b - 1) / b, (n + b - 1) / b);
    if (opts->resume_steps < 0 || opts->resume_steps > steps) { set_arg_error(16); return RRF_INVALID_ARG; }
    if (opts->resume_steps > 0 && (m < n || opts->oversample != 0 || opts->q_policy != RRF_Q_FIXED)) {
      set_arg_error(16);
      return RRF_INVALID_ARG;
    }
    if (opts->oversample < 0 || b + opts->oversample > 256) { set_arg_error(16); return RRF_INVALID_ARG; }
    if (!(opts->frob_tol >= 0.0) || std::isinf(opts->frob_tol)) { set_arg_error(16); return RRF_INVALID_ARG; }
    if (opts->oversample > 0 && (opts->sketch_prec != RRF_SKETCH_FP64 || opts->reorth != 0 ||
                                 opts->q_policy != RRF_Q_FIXED)) {
      set_arg_error(16);
      return RRF_INVALID_ARG;
    }
    if (opts->gemm_mode < RRF_GEMM_AUTO || opts->gemm_mode > RRF_GEMM_EMULATED) { set_arg_error(16); return RRF_INVALID_ARG; }
    if (opts->q_per_block != nullptr) {
      for (int64_t i = 0; i < steps; ++i)
        if (opts->q_per_block[i] < 0 || opts->q_per_block[i] > 16) { set_arg_error(16); return RRF_INVALID_ARG; }
    }
  }
  return RRF_OK;
}

}  // namespace
}  // namespace rrf

using namespace rrf;

extern "C" size_t rrf_randutv_workspace(int64_t m, int64_t n, int64_t b, const rrf_opts* opts) {
  if (m < 1 || n < 1 || b < 1) return 0;
  if (m < n) return wide_workspace(rrf_randutv_workspace, m, n, b, opts);
  Arena ar;
  RWs w;
  const bool bf16 = opts != nullptr && opts->sketch_prec == RRF_SKETCH_BF16;
  const int64_t p = opts != nullptr ? std::max(opts->oversample, 0) : 0;
  return layout(m, n, b, p, bf16, opts ? opts->gemm_mode : RRF_GEMM_AUTO, ar, w);
}

extern "C" rrf_status rrf_randutv(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int q,
                                  double* U, int64_t ldu, double* T, int64_t ldt, double* V, int64_t ldv,
                                  uint64_t seed, void* workspace, size_t ws_bytes, const rrf_opts* opts,
                                  void* stream_) {
  if (m >= 1 && n > m)  // wide: factor A^T and transpose the result
    return factor_wide(rrf_randutv_workspace, rrf_randutv, m, n, A, lda, b, q, U, ldu, T, ldt, V, ldv, seed,
                       workspace, ws_bytes, opts, stream_);
  rrf_status st = check_args(m, n, A, lda, b, q, U, ldu, T, ldt, V, ldv, opts);
  if (st != RRF_OK) return st;
  const bool bf16 = opts != nullptr && opts->sketch_prec == RRF_SKETCH_BF16;
  const bool reorth = bf16 || (opts != nullptr && opts->reorth != 0);
  const size_t need = rrf_randutv_workspace(m, n, b, opts);
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0) {
    set_arg_error(14);
    return RRF_INVALID_ARG;
  }
  if (ws_bytes < need) {
    set_arg_error(15);
    return RRF_WORKSPACE_TOO_SMALL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  Arena ar;
  ar.base = reinterpret_cast<char*>(workspace);
  ar.cap = ws_bytes;
  RWs w;
  const int64_t p = opts != nullptr ? opts->oversample : 0;
  layout(m, n, b, p, bf16, opts ? opts->gemm_mode : RRF_GEMM_AUTO, ar, w);
  if (ar.overflow) return RRF_WORKSPACE_TOO_SMALL;

  RRF_CUDA_TRY(cudaMemsetAsync(w.hdr, 0, kHeaderBytes, s));
  // Resume: U, T, V already hold the factorization after `start` steps; A is not read.
  const int64_t start = opts != nullptr ? opts->resume_steps : 0;
  if (start == 0) {
    RRF_CUDA_TRY(check_finite(m, n, A, lda, &w.hdr->status, s));
    // T = A (nothing to copy when factoring in place); U = I_m; V = I_n.
    if (T != A) RRF_CUDA_TRY(copy_matrix(m, n, A, lda, T, ldt, s));
    RRF_CUDA_TRY(fill_identity(m, m, U, ldu, s));
    RRF_CUDA_TRY(fill_identity(n, n, V, ldv, s));
  }

  const int64_t steps = std::min((m + b - 1) / b, (n + b - 1) / b);
  const bool learned = opts != nullptr && opts->q_policy == RRF_Q_LEARNED;
  bool have_next = false;  // randUTV_boosted: W_next of the previous step is in w.Wn
  // Early termination (Sec. 4.1): e_0 = ||A||_F, then the recurrence after every step.
  const double frob_tol = opts != nullptr ? opts->frob_tol : 0.0;
  const bool frob = opts != nullptr && (frob_tol > 0.0 || opts->frob_out != nullptr);
  auto below_tol = [&](int64_t idx, bool* stop) -> cudaError_t {
    double e2 = 0.0;
    cudaError_t e = cudaMemcpyAsync(&e2, w.e2 + idx, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *stop = e2 <= frob_tol * frob_tol;
    return e;
  };
  bool stop = false;
  int64_t done = start;
  int* fgate = &w.hdr->flags[8];  // set when the recurrence fell below its accuracy floor
  // The b x b SVD of step i runs on a side stream while the main stream applies U_i and samples step i + 1
  // (their data are disjoint from R's SVD); its small updates then run on the main stream just before
  // V_{i+1} is applied -- the first operation that touches what they write (the row block T(I2, J3)) --
  // so every element sees the same operations in the same order as in the serial schedule, and the result
  // is the same bit for bit.  Not with the learned policy (its features wait for the SVD) or a Frobenius
  // tolerance (the stop test waits for the small updates), nor for b > 128.
  SideStream* side = (!learned && frob_tol == 0.0 && b <= 128) ? side_stream() : nullptr;
  RRF_CUDA_TRY(cudaMemsetAsync(w.hdr2, 0, kHeaderBytes, s));
  struct Pend {
    bool on;
    int64_t i, o, r, c;
    int par;
  } pend = {false, 0, 0, 0, 0, 0};
  // U(:, I2) U_small, V(:, J2) V_small, U_small^T T(I2, J3), T(I1, J2) V_small, T(I2 u I3, J2) = [D; 0] of the
  // pending step, then its Frobenius recurrence.
  auto small_updates = [&]() -> cudaError_t {
    const int64_t o = pend.o, r = pend.r, c = pend.c, nc = c - b;
    const double* Usp = pend.par ? w.Us1 : w.Us;
    const double* Vsp = pend.par ? w.Vs1 : w.Vs;
    const double* sgp = pend.par ? w.sig1 : w.sig;
    double* T22p = T + o + o * ldt;
    double* UI2 = U + o * ldu;
    double* VJ2 = V + o * ldv;
    double* TI2J3 = T + o + (o + b) * ldt;
    double* TI1J2 = T + o * ldt;
    pend.on = false;
    GemmDesc g[4] = {gd(m, b, b, UI2, ldu, 0, Usp, b, 0, w.Xa, m),
                     gd(n, b, b, VJ2, ldv, 0, Vsp, b, 0, w.Xb, n),
                     gd(b, nc, b, Usp, b, 1, TI2J3, ldt, 0, w.Wa, b),
                     gd(o, b, b, TI1J2, ldt, 0, Vsp, b, 0, w.Xc, std::max<int64_t>(o, 1))};
    cudaError_t e = gemm_run(w.eng, g, o > 0 ? 4 : 3, s);
    if (e == cudaSuccess) e = copy_matrix(m, b, w.Xa, m, UI2, ldu, s);
    if (e == cudaSuccess) e = copy_matrix(n, b, w.Xb, n, VJ2, ldv, s);
    if (e == cudaSuccess) e = copy_matrix(b, nc, w.Wa, b, TI2J3, ldt, s);
    if (e == cudaSuccess && o > 0) e = copy_matrix(o, b, w.Xc, o, TI1J2, ldt, s);
    if (e == cudaSuccess) e = set_diag_block(r, b, sgp, T22p, ldt, s);
    if (e == cudaSuccess && frob) {  // e_i^2 = e_{i-1}^2 - ||T(I2, J2 u J3)||_F^2; direct below the floor
      e = frob_step(b, c, T22p, ldt, w.fpart, w.e2, pend.i, false, start, fgate, s);
      if (e == cudaSuccess) e = frob_refresh(r - b, c - b, T22p + b + b * ldt, ldt, w.fpart, w.e2, pend.i, fgate, s);
    }
    return e;
  };
  auto flush = [&]() -> cudaError_t {
    if (!pend.on) return cudaSuccess;
    if (side != nullptr) {
      cudaError_t e = cudaStreamWaitEvent(s, side->ev_j[pend.par], 0);
      if (e != cudaSuccess) return e;
      w.eng.max_ctas = 0;
    }
    return small_updates();
  };
  if (frob) {  // e_start from its definition: ||A||_F, or the trailing block's norm when resuming
    const int64_t o = b * start;
    if (start == 0) RRF_CUDA_TRY(frob_step(m, n, A, lda, w.fpart, w.e2, 0, true, 0, fgate, s));
    else RRF_CUDA_TRY(frob_step(m - o, n - o, T + o + o * ldt, ldt, w.fpart, w.e2, start, true, start, fgate, s));
    if (frob_tol > 0.0) RRF_CUDA_TRY(below_tol(start, &stop));
  }
  for (int64_t i = start + 1; i <= steps && !stop; ++i) {
    const int64_t o = b * (i - 1);
    const int64_t r = m - o, c = n - o;
    double* T22 = T + o + o * ldt;
    if (b * i < m && b * i < n) {
      int qi = (opts != nullptr && opts->q_per_block != nullptr) ? opts->q_per_block[i - 1] : q;
      const int64_t pk = std::min(p, c - b);  // oversampling of this step (fewer columns near the end)
      if (p > 0) {
        // randUTV_boosted: sample of b + pk columns; V_i from its leading b left singular vectors.
        if (opts->q_used_out != nullptr) opts->q_used_out[i - 1] = qi;
        RRF_CUDA_TRY(boosted_sample(i, r, c, b, pk, i > 1 && have_next, qi, T22, ldt, seed, w, s));
        RRF_CUDA_TRY(boosted_svd(c, b, b + pk, w, s));
      } else {
        // randUTV_basic sketch.
        RRF_CUDA_TRY(randn_f64(r, b, w.G, r, seed, (uint32_t)i, 1u, s));
        RRF_CUDA_TRY(sketch_begin(r, c, b, T22, ldt, bf16, w, s));
        const double* start = nullptr;
        if (learned) {
          // Features from the q = 0 sketch (the R of its Householder QR), MLP -> q for this step.
          RRF_CUDA_TRY(copy_matrix(c, b, w.Y, c, w.Qt, c, s));
          RRF_CUDA_TRY(panel_qr(c, b, w.Qt, c, w.tauv, w.Yv, c, w.Tv, b, nullptr, 0, w.panel, w.panel_bytes, w.hdr,
                                s, &w.eng));
          RRF_CUDA_TRY(policy_features(w.Qt, c, (int)b, i > 1 ? w.sig : nullptr, (int)i, (int)steps, n, c, w.feat,
                                       s));
          if (opts->mlp_params != nullptr) {
            RRF_CUDA_TRY(policy_decide(opts->mlp_params, w.feat, w.qdev, s));
            int qh = q;
            RRF_CUDA_TRY(cudaMemcpyAsync(&qh, w.qdev, sizeof(int), cudaMemcpyDeviceToHost, s));
            if (opts->features_out != nullptr)
              RRF_CUDA_TRY(cudaMemcpyAsync(opts->features_out + 16 * (i - 1), w.feat, 16 * sizeof(float),
                                           cudaMemcpyDeviceToHost, s));
            RRF_CUDA_TRY(cudaStreamSynchronize(s));
            qi = qh;
          } else if (opts->features_out != nullptr) {
            RRF_CUDA_TRY(cudaMemcpyAsync(opts->features_out + 16 * (i - 1), w.feat, 16 * sizeof(float),
                                         cudaMemcpyDeviceToHost, s));
            RRF_CUDA_TRY(cudaStreamSynchronize(s));
          }
          if (reorth && qi > 0) {  // the QR just computed gives the orthonormal start for free
            RRF_CUDA_TRY(explicit_q(c, b, w.Yv, w.Tv, w.Wkk, w.Qt, w, s));
            start = w.Qt;
          }
        }
        if (opts != nullptr && opts->q_used_out != nullptr) opts->q_used_out[i - 1] = qi;
        RRF_CUDA_TRY(sketch_continue(r, c, b, T22, ldt, qi, bf16, reorth, start, w, s));
      }
      // V_i = I - Yv Tv Yv^T from HQR_full(Y); T(:, o:) and V(:, o:) <- (.) V_i.
      RRF_CUDA_TRY(panel_qr(c, b, w.Y, c, w.tauv, w.Yv, c, w.Tv, b, nullptr, 0, w.panel, w.panel_bytes,
                            w.hdr, s, &w.eng));
      // The previous step's small updates go first: its row block T(I2, J3) meets this V_i next.
      RRF_CUDA_TRY(flush());
      {
        double* CT = T + o * ldt;
        double* CV = V + o * ldv;
        GemmDesc g1[2] = {gd(m, b, c, CT, ldt, 0, w.Yv, c, 0, w.Xa, m),
                          gd(n, b, c, CV, ldv, 0, w.Yv, c, 0, w.Xb, n)};
        RRF_CUDA_TRY(gemm_run(w.eng, g1, 2, s));
        GemmDesc g2[2] = {gd(m, b, b, w.Xa, m, 0, w.Tv, b, 0, w.Xc, m),
                          gd(n, b, b, w.Xb, n, 0, w.Tv, b, 0, w.Xd, n)};
        RRF_CUDA_TRY(gemm_run(w.eng, g2, 2, s));
        GemmDesc g3[2] = {gd(m, c, b, w.Xc, m, 0, w.Yv, c, 1, CT, ldt, -1.0, 1.0),
                          gd(n, c, b, w.Xd, n, 0, w.Yv, c, 1, CV, ldv, -1.0, 1.0)};
        RRF_CUDA_TRY(gemm_run(w.eng, g3, 2, s));
      }
      if (p > 0) {
        RRF_CUDA_TRY(boosted_next(c, b, pk, w, s));
        have_next = pk > 0;
      }
      // [U_i, R] = HQR_full(T(o:, o:o+b)); R goes to this step's parity buffer.
      const int par = (int)(i & 1);
      double* Rp = par ? w.Rs1 : w.Rs;
      RRF_CUDA_TRY(panel_qr(r, b, T22, ldt, w.tauu, w.Yu, r, w.Tu, b, Rp, b, w.panel, w.panel_bytes,
                            w.hdr, s, &w.eng));
      if (side != nullptr) {
        // SVD of R on the side stream, beside U_i's application and the next step's sample; the main
        // stream keeps kSideReserve SMs free for it until it waits for the result.
        RRF_CUDA_TRY(cudaEventRecord(side->ev_r[par], s));
        RRF_CUDA_TRY(cudaStreamWaitEvent(side->s, side->ev_r[par], 0));
        RRF_CUDA_TRY(jacobi_svd(b, Rp, b, par ? w.Us1 : w.Us, b, par ? w.sig1 : w.sig, par ? w.Vs1 : w.Vs, b, w.hdr2,
                                side->s, w.jscr, w.jscr_bytes));
        RRF_CUDA_TRY(cudaEventRecord(side->ev_j[par], side->s));
        w.eng.max_ctas = std::max(1, dev_info().sms - kSideReserve);
        pend = {true, i, o, r, c, par};
      }
      {
        double* C = T + o + (o + b) * ldt;  // r x (c - b)
        double* CU = U + o * ldu;           // m x r
        const int64_t nc = c - b;
        GemmDesc g1[2] = {gd(b, nc, r, w.Yu, r, 1, C, ldt, 0, w.Wa, b),
                          gd(m, b, r, CU, ldu, 0, w.Yu, r, 0, w.Xa, m)};
        RRF_CUDA_TRY(gemm_run(w.eng, g1, 2, s));
        GemmDesc g2[2] = {gd(b, nc, b, w.Tu, b, 1, w.Wa, b, 0, w.Wb, b),
                          gd(m, b, b, w.Xa, m, 0, w.Tu, b, 0, w.Xc, m)};
        RRF_CUDA_TRY(gemm_run(w.eng, g2, 2, s));
        GemmDesc g3[2] = {gd(r, nc, b, w.Yu, r, 0, w.Wb, b, 0, C, ldt, -1.0, 1.0),
                          gd(m, r, b, w.Xc, m, 0, w.Yu, r, 1, CU, ldu, -1.0, 1.0)};
        RRF_CUDA_TRY(gemm_run(w.eng, g3, 2, s));
      }
      if (side == nullptr) {
        // SVD of R and the small updates, in order.  The same SVD kernel (cluster size and pre-pass) as on
        // the side stream, so both schedules give the same bits.
        RRF_CUDA_TRY(jacobi_svd(b, Rp, b, w.Us, b, w.sig, w.Vs, b, w.hdr, s, w.gemm, w.gemm_bytes));
        pend = {true, i, o, r, c, 0};
        RRF_CUDA_TRY(small_updates());
        if (frob_tol > 0.0) RRF_CUDA_TRY(below_tol(i, &stop));
      }
    } else {
      // Final block: SVD of the r x c remainder (c <= b).
      RRF_CUDA_TRY(flush());
      const double* M = T22;
      int64_t ldm = ldt;
      if (r > c) {
        RRF_CUDA_TRY(panel_qr(r, c, T22, ldt, w.tauu, w.Yu, r, w.Tu, c, w.Rs, c, w.panel, w.panel_bytes,
                              w.hdr, s, &w.eng));
        M = w.Rs;
        ldm = c;
      }
      RRF_CUDA_TRY(jacobi_svd(c, M, ldm, w.Us, c, w.sig, w.Vs, c, w.hdr, s, w.gemm, w.gemm_bytes));
      double* CU = U + o * ldu;
      if (r > c) {  // U(:, o:) <- U(:, o:) (I - Yu Tu Yu^T)
        GemmDesc g1 = gd(m, c, r, CU, ldu, 0, w.Yu, r, 0, w.Xa, m);
        RRF_CUDA_TRY(gemm_run(w.eng, &g1, 1, s));
        GemmDesc g2 = gd(m, c, c, w.Xa, m, 0, w.Tu, c, 0, w.Xc, m);
        RRF_CUDA_TRY(gemm_run(w.eng, &g2, 1, s));
        GemmDesc g3 = gd(m, r, c, w.Xc, m, 0, w.Yu, r, 1, CU, ldu, -1.0, 1.0);
        RRF_CUDA_TRY(gemm_run(w.eng, &g3, 1, s));
      }
      double* VJ = V + o * ldv;
      double* TI1J = T + o * ldt;
      GemmDesc g[3] = {gd(m, c, c, CU, ldu, 0, w.Us, c, 0, w.Xa, m),
                       gd(n, c, c, VJ, ldv, 0, w.Vs, c, 0, w.Xb, n),
                       gd(o, c, c, TI1J, ldt, 0, w.Vs, c, 0, w.Xc, std::max<int64_t>(o, 1))};
      RRF_CUDA_TRY(gemm_run(w.eng, g, o > 0 ? 3 : 2, s));
      RRF_CUDA_TRY(copy_matrix(m, c, w.Xa, m, CU, ldu, s));
      RRF_CUDA_TRY(copy_matrix(n, c, w.Xb, n, VJ, ldv, s));
      if (o > 0) RRF_CUDA_TRY(copy_matrix(o, c, w.Xc, o, TI1J, ldt, s));
      RRF_CUDA_TRY(set_diag_block(r, c, w.sig, T22, ldt, s));
      if (frob) RRF_CUDA_TRY(cudaMemsetAsync(w.e2 + i, 0, sizeof(double), s));  // nothing left
    }
    done = i;
  }
  RRF_CUDA_TRY(flush());
  if (side != nullptr) RRF_CUDA_TRY(merge_status(&w.hdr->status, &w.hdr2->status, s));
  if (opts != nullptr && opts->steps_out != nullptr) *opts->steps_out = (int)done;
  if (opts != nullptr && opts->frob_out != nullptr) {
    std::vector<double> e2((size_t)done + 1);
    RRF_CUDA_TRY(cudaMemcpyAsync(e2.data(), w.e2, e2.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    RRF_CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t j = 0; j < e2.size(); ++j) opts->frob_out[j] = (int64_t)j < start ? NAN : std::sqrt(e2[j]);
  }
  return RRF_OK;
}
