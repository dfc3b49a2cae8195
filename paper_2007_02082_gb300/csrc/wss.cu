// Wall shear stress at the Lagrangian points (Sec. 2.6): WSS = |t - (t.n) n|,
// t = 2 mu eps(u) n, with the velocity derivatives from second-order DC-PSE
// operators (the meshless method Sec. 2.6 cites) over the finest-level nodes
// around each wall point on the fluid side.  One thread per wall point, FP64.
#include <algorithm>
#include <cmath>

#include "device.cuh"
#include "ibmove.hpp"
#include "wss.hpp"

namespace ibg {

IBG_KCOUNT_DEFINE
unsigned long long wss_kcount() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, g_kcount, sizeof(v));
  return v;
}

namespace {

// the nine monomials z^alpha, 1 <= |alpha| <= 2, first-degree ones first
__device__ __forceinline__ void monomials(const double z[3], double P[9]) {
  P[0] = z[0];
  P[1] = z[1];
  P[2] = z[2];
  P[3] = z[0] * z[0];
  P[4] = z[0] * z[1];
  P[5] = z[0] * z[2];
  P[6] = z[1] * z[1];
  P[7] = z[1] * z[2];
  P[8] = z[2] * z[2];
}

// Candidate q of point p: a finest-level node within the cutoff on the fluid
// side.  Distances and projections are rounded term by term (no fused
// multiply-add) so that the selection is exactly that of a plain evaluation.
struct Cand {
  const MoveGrid& G;
  const double* Xp;
  const double* np_;
  double rc2;
  __device__ bool operator()(const int64_t q[3], int32_t& slot, double d[3]) const {
    const int64_t bx = q[0] / DBS, by = q[1] / DBS, bz = q[2] / DBS;
    const int32_t b = G.bmap[(bz * G.nb[1] + by) * G.nb[0] + bx];
    if (b < 0) return false;
    const int64_t s = (int64_t)b * DBV + ((q[2] % DBS) * DBS + (q[1] % DBS)) * DBS + (q[0] % DBS);
    if (!(G.meta[s] & D_VALID)) return false;
    for (int a = 0; a < 3; ++a) d[a] = __dsub_rn(__dadd_rn(G.origin[a], __dmul_rn(double(q[a]), G.hf[a])), Xp[a]);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
    if (!(r2 <= rc2)) return false;
    const double dn = __dadd_rn(__dadd_rn(__dmul_rn(d[0], np_[0]), __dmul_rn(d[1], np_[1])), __dmul_rn(d[2], np_[2]));
    if (!(dn < 0.0)) return false;
    slot = int32_t(s);
    return true;
  }
};

__global__ void k_wss(MoveGrid G, int64_t M, const double* __restrict__ X, const double* __restrict__ UB,
                      const double* __restrict__ nrm, const double* __restrict__ u, int64_t ns, double eps,
                      double rc2, int32_t rx, int32_t ry, int32_t rz, double mu2, double* __restrict__ wss,
                      double* __restrict__ grad, int32_t* __restrict__ err) {
  KCOUNT();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= M) return;
  const double* Xp = X + 3 * p;
  const double* np_ = nrm + 3 * p;
  const int32_t rad[3] = {rx, ry, rz};
  int64_t lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    const int64_t c = int64_t(floor((Xp[a] - G.origin[a]) / G.hf[a]));
    lo[a] = c - rad[a] < 0 ? 0 : c - rad[a];
    hi[a] = c + 1 + rad[a] > G.nf[a] ? G.nf[a] : c + 1 + rad[a];
  }
  const Cand cand{G, Xp, np_, rc2};
  // moment matrix A = sum_q w_q P_q P_q^T (lower triangle, row-major packed)
  double A[45];
  for (int k = 0; k < 45; ++k) A[k] = 0.0;
  int32_t n = 0;
  int64_t q[3];
  for (q[2] = lo[2]; q[2] <= hi[2]; ++q[2])
    for (q[1] = lo[1]; q[1] <= hi[1]; ++q[1])
      for (q[0] = lo[0]; q[0] <= hi[0]; ++q[0]) {
        int32_t s;
        double d[3];
        if (!cand(q, s, d)) continue;
        const double z[3] = {d[0] / eps, d[1] / eps, d[2] / eps};
        double P[9];
        monomials(z, P);
        const double w = exp(-(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]));
        int k = 0;
        for (int r = 0; r < 9; ++r)
          for (int c = 0; c <= r; ++c) A[k++] += w * P[r] * P[c];
        ++n;
      }
  // Cholesky A = L L^T in place, then coef[:, j] = A^-1 e_j for j = 0, 1, 2
  bool ok = n >= 9;
  for (int r = 0; r < 9 && ok; ++r) {
    for (int c = 0; c <= r; ++c) {
      double v = A[r * (r + 1) / 2 + c];
      for (int k = 0; k < c; ++k) v -= A[r * (r + 1) / 2 + k] * A[c * (c + 1) / 2 + k];
      if (c == r) {
        if (!(v > 0.0)) { ok = false; break; }
        A[r * (r + 1) / 2 + r] = sqrt(v);
      } else {
        A[r * (r + 1) / 2 + c] = v / A[c * (c + 1) / 2 + c];
      }
    }
  }
  if (!ok) {
    atomicMax(err, 1);
    wss[p] = 0.0;
    return;
  }
  double coef[3][9];
  for (int j = 0; j < 3; ++j) {
    double y[9];
    for (int r = 0; r < 9; ++r) {   // L y = e_j
      double v = r == j ? 1.0 : 0.0;
      for (int k = 0; k < r; ++k) v -= A[r * (r + 1) / 2 + k] * y[k];
      y[r] = v / A[r * (r + 1) / 2 + r];
    }
    for (int r = 8; r >= 0; --r) {   // L^T x = y
      double v = y[r];
      for (int k = r + 1; k < 9; ++k) v -= A[k * (k + 1) / 2 + r] * coef[j][k];
      coef[j][r] = v / A[r * (r + 1) / 2 + r];
    }
  }
  // d u_i / d x_j = (1/eps) sum_q (u_i(q) - U_B,i) eta_j(z_q)
  double g[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (q[2] = lo[2]; q[2] <= hi[2]; ++q[2])
    for (q[1] = lo[1]; q[1] <= hi[1]; ++q[1])
      for (q[0] = lo[0]; q[0] <= hi[0]; ++q[0]) {
        int32_t s;
        double d[3];
        if (!cand(q, s, d)) continue;
        const double z[3] = {d[0] / eps, d[1] / eps, d[2] / eps};
        double P[9];
        monomials(z, P);
        const double w = exp(-(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]));
        double eta[3];
        for (int j = 0; j < 3; ++j) {
          double v = 0.0;
          for (int r = 0; r < 9; ++r) v += P[r] * coef[j][r];
          eta[j] = w * v;
        }
        for (int i = 0; i < 3; ++i) {
          const double du = u[(int64_t)i * ns + s] - UB[3 * p + i];
          for (int j = 0; j < 3; ++j) g[i][j] += du * eta[j];
        }
      }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) g[i][j] /= eps;
  // t = 2 mu eps(u) n with eps(u) = (g + g^T) / 2
  double t[3];
  for (int i = 0; i < 3; ++i) {
    double v = 0.0;
    for (int j = 0; j < 3; ++j) v += 0.5 * (g[i][j] + g[j][i]) * np_[j];
    t[i] = mu2 * v;
  }
  const double tn = t[0] * np_[0] + t[1] * np_[1] + t[2] * np_[2];
  double s2 = 0.0;
  for (int i = 0; i < 3; ++i) {
    const double v = t[i] - tn * np_[i];
    s2 += v * v;
  }
  wss[p] = sqrt(s2);
  if (grad)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) grad[9 * p + 3 * i + j] = g[i][j];
}

}  // namespace

void wss_compute(const MoveGrid& G, const double hf[3], int64_t M, const double* X, const double* UB,
                 const double* nrm, const double* u, int64_t ns, double nu_rho, double* wss, double* grad,
                 int32_t* err, cudaStream_t st) {
  if (M == 0) return;
  const double e = std::max(hf[0], std::max(hf[1], hf[2]));
  const double rc = WSS_RADIUS * e;
  int32_t r[3];
  for (int a = 0; a < 3; ++a) r[a] = int32_t(std::ceil(rc / hf[a])) + 1;
  IBG_LAUNCH(k_wss, unsigned((M + 63) / 64), 64, 0, st, G, M, X, UB, nrm, u, ns, e, rc * rc, r[0], r[1], r[2],
             2.0 * nu_rho, wss, grad, err);
}

}  // namespace ibg
