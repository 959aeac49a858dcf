// Per-particle mass matrices (Sec. 5, "Exploitation of local geometry"): at
// the start of a stage every particle gets M = beta F(theta) + prior Hessian +
// 12 / width^2 on the diagonal, F the Fisher information of the Whittle
// likelihood (the Gauss-Newton part of -d^2 ln L, positive semi-definite), and
// keeps it through the stage's mutation.
//
// With the Newtonian amplitude every strain derivative is the strain times a
// function of frequency that is linear in the phase basis:
//   d_j h_a(f) = (d_j G_a - 2 pi i G_a phi_aj(f)) A(f) e^{-i Psi_a(f)},
//   phi_aj(f) = sum_m D_ajm B_m(f),  B = {x^5, x^3, x^2, x, ln f, y, y ln f, y^2, f, 1},
// so <d_j h_a | d_k h_a> needs only prefix sums over the bins below f_ISCO of
// W = w f^-7/3 times 1, B_m and B_m B_n (tables built once per event):
//   F_jk = sum_a Re(conj(dG_j) dG_k) P0 - 2 pi [Im(conj(G) dG_j) (D_k . P1)
//          + Im(conj(G) dG_k) (D_j . P1)] + 4 pi^2 |G|^2 D_j P2 D_k.
// FP64 throughout (the entries span many decades in physical units).
#include <cmath>
#include <vector>

#include "context.cuh"
#include "physics.cuh"

using namespace sharpy;

namespace sharpy {

constexpr int kNB = kNBasis + 1;  // basis incl. the constant
constexpr int kNPair = kNBasis * (kNBasis + 1) / 2;

__device__ __forceinline__ int pair_index(int m, int n) {  // m <= n < kNBasis
  return m * kNBasis - m * (m - 1) / 2 + (n - m);
}

// Prefix sums (basis-weighted) at the last active bin.
__device__ void fisher_sums(const DevEvent& ev, int a, int k, double* P1, double (*P2)[kNB]) {
  const int64_t K = ev.n_bins;
  const double P0 = ev.pref[(int64_t)a * K + k];
  for (int m = 0; m < kNBasis; ++m) P1[m] = ev.p1[((int64_t)a * kNBasis + m) * K + k];
  P1[kNBasis] = P0;
  for (int m = 0; m < kNBasis; ++m)
    for (int n = m; n < kNBasis; ++n) {
      const double v = ev.p2[((int64_t)a * kNPair + pair_index(m, n)) * K + k];
      P2[m][n] = v;
      P2[n][m] = v;
    }
  for (int m = 0; m < kNBasis; ++m) P2[m][kNBasis] = P2[kNBasis][m] = P1[m];
  P2[kNBasis][kNBasis] = P0;
}

// F over the eleven physical parameters (GW model).
__device__ void fisher_phys(const DevModel& m, const DevEvent& ev, const double* x, double (*F)[SHARPY_NPHYS]) {
  for (int j = 0; j < SHARPY_NPHYS; ++j)
    for (int l = 0; l < SHARPY_NPHYS; ++l) F[j][l] = 0.0;
  SweepCoef sc;
  EpiCoef<double> ec;
  prologue<double, true>(m, ev, x, sc, ec);
  if (!sc.ok || sc.kisco < 0) return;
  for (int a = 0; a < ev.n_det; ++a) {
    double P1[kNB], P2[kNB][kNB];
    fisher_sums(ev, a, sc.kisco, P1, P2);
    const double P0 = P1[kNBasis];
    const double A0 = ec.A0;
    const double Gr = A0 * ec.cre[a], Gi = A0 * ec.cim[a];
    // dG_j (complex) and the phase-basis Jacobian D_j
    double dGr[SHARPY_NPHYS], dGi[SHARPY_NPHYS], Dj[SHARPY_NPHYS][kNB];
    for (int j = 0; j < SHARPY_NPHYS; ++j) {
      dGr[j] = dGi[j] = 0.0;
      for (int b = 0; b < kNB; ++b) Dj[j][b] = 0.0;
    }
    const int pn[4] = {SHARPY_MC, SHARPY_Q, SHARPY_CHI1, SHARPY_CHI2};
    for (int p = 0; p < 4; ++p) {
      for (int b = 0; b < kNPn; ++b) Dj[pn[p]][b] = ec.dalpha[b][p];
      Dj[pn[p]][kNBasis] = ec.dc0[p];
    }
    dGr[SHARPY_MC] = Gr * ec.rel_mc;
    dGi[SHARPY_MC] = Gi * ec.rel_mc;
    dGr[SHARPY_DL] = Gr * ec.rel_dl;
    dGi[SHARPY_DL] = Gi * ec.rel_dl;
    const int resp[4] = {SHARPY_COSI, SHARPY_PSI, SHARPY_RA, SHARPY_SINDEC};
    for (int r = 0; r < 4; ++r) {
      dGr[resp[r]] = A0 * ec.dcre[a][r];
      dGi[resp[r]] = A0 * ec.dcim[a][r];
    }
    Dj[SHARPY_PHIC][kNBasis] = -1.0 / kTwoPi;
    Dj[SHARPY_TC][kNPn] = 1.0;
    Dj[SHARPY_RA][kNPn] = ec.dtau[a][0];
    Dj[SHARPY_SINDEC][kNPn] = ec.dtau[a][1];
    double dp1[SHARPY_NPHYS], img[SHARPY_NPHYS];
    for (int j = 0; j < SHARPY_NPHYS; ++j) {
      double t = 0.0;
      for (int b = 0; b < kNB; ++b) t += Dj[j][b] * P1[b];
      dp1[j] = t;
      img[j] = Gr * dGi[j] - Gi * dGr[j];  // Im(conj(G) dG_j)
    }
    const double g2 = Gr * Gr + Gi * Gi;
    for (int j = 0; j < SHARPY_NPHYS; ++j) {
      double row[kNB];
      for (int c = 0; c < kNB; ++c) {
        double t = 0.0;
        for (int b = 0; b < kNB; ++b) t += Dj[j][b] * P2[b][c];
        row[c] = t;
      }
      for (int l = j; l < SHARPY_NPHYS; ++l) {
        double q = 0.0;
        for (int c = 0; c < kNB; ++c) q += row[c] * Dj[l][c];
        const double v = (dGr[j] * dGr[l] + dGi[j] * dGi[l]) * P0 - kTwoPi * (img[j] * dp1[l] + img[l] * dp1[j]) +
                         kTwoPi * kTwoPi * g2 * q;
        F[j][l] += v;
        if (l != j) F[l][j] += v;
      }
    }
  }
}

// Cholesky M = C C^T in place (lower triangle); false if not positive definite.
__device__ bool cholesky(double (*M)[kMaxDim], int D) {
  for (int j = 0; j < D; ++j) {
    double d = M[j][j];
    for (int k = 0; k < j; ++k) d -= M[j][k] * M[j][k];
    if (!(d > 0.0) || !isfinite(d)) return false;
    const double c = sqrt(d);
    M[j][j] = c;
    for (int i = j + 1; i < D; ++i) {
      double t = M[i][j];
      for (int k = 0; k < j; ++k) t -= M[i][k] * M[j][k];
      M[i][j] = t / c;
    }
  }
  for (int i = 0; i < D; ++i)
    for (int j = i + 1; j < D; ++j) M[i][j] = 0.0;
  return true;
}

__global__ void local_metric_kernel(DevModel m, DevEvent ev, int64_t n, const double* __restrict__ theta,
                                    const double* beta_ptr, double beta_val, double* mass, double* minv, double* chol,
                                    int* status) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int D = m.n_dim;
  const double beta = beta_ptr ? *beta_ptr : beta_val;
  double x[kMaxDim];
  for (int i = 0; i < D; ++i) x[i] = theta[p * D + i];
  double M[kMaxDim][kMaxDim];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) M[i][j] = 0.0;
  if (m.model == SHARPY_MODEL_TAYLORF2) {
    double F[SHARPY_NPHYS][SHARPY_NPHYS];
    fisher_phys(m, ev, x, F);
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) M[i][j] = beta * F[m.phys[i]][m.phys[j]];
  } else {
    // mixture: responsibility-weighted component precisions
    double lc[SHARPY_MAX_COMP], best = -INFINITY;
    for (int c = 0; c < m.n_comp; ++c) {
      double t = m.mix_logw[c];
      for (int i = 0; i < D; ++i) {
        const double z = (x[i] - m.mix_mu[c][i]) / m.mix_sigma[c][i];
        t += -0.5 * z * z - log(m.mix_sigma[c][i]);
      }
      lc[c] = t;
      best = fmax(best, t);
    }
    double tot = 0.0;
    for (int c = 0; c < m.n_comp; ++c) tot += exp(lc[c] - best);
    for (int c = 0; c < m.n_comp; ++c) {
      const double r = exp(lc[c] - best) / tot;
      for (int i = 0; i < D; ++i) M[i][i] += beta * r / (m.mix_sigma[c][i] * m.mix_sigma[c][i]);
    }
  }
  for (int i = 0; i < D; ++i) {
    const double w = m.hi[i] - m.lo[i];
    M[i][i] += 12.0 / (w * w);
    if (m.prior[i] == SHARPY_PRIOR_POWER2) M[i][i] += 2.0 / (x[i] * x[i]);
  }
  if (mass)
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) mass[(p * D + i) * D + j] = M[i][j];
  if (!minv && !chol) return;
  // M^-1 = C^-T C^-1 with M = C C^T; then L L^T = M^-1 (lower L)
  double C[kMaxDim][kMaxDim];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) C[i][j] = M[i][j];
  if (!cholesky(C, D)) {
    // not positive definite in floating point: keep the diagonal (positive by construction)
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) C[i][j] = i == j ? sqrt(M[i][i]) : 0.0;
  }
  double Ci[kMaxDim][kMaxDim];  // C^-1 (lower)
  for (int j = 0; j < D; ++j) {
    for (int i = 0; i < D; ++i) Ci[i][j] = 0.0;
    Ci[j][j] = 1.0 / C[j][j];
    for (int i = j + 1; i < D; ++i) {
      double t = 0.0;
      for (int k = j; k < i; ++k) t -= C[i][k] * Ci[k][j];
      Ci[i][j] = t / C[i][i];
    }
  }
  double Mi[kMaxDim][kMaxDim];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      double t = 0.0;
      for (int k = (i > j ? i : j); k < D; ++k) t += Ci[k][i] * Ci[k][j];
      Mi[i][j] = t;
    }
  if (minv)
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) minv[(p * D + i) * D + j] = Mi[i][j];
  if (chol) {
    if (!cholesky(Mi, D))
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) Mi[i][j] = i == j ? 1.0 / C[i][i] : 0.0;
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) chol[(p * D + i) * D + j] = Mi[i][j];
  }
}

// Build the Fisher prefix tables of the staged event (host, compensated sums).
int ensure_fisher_tables(sharpy_ctx* c) {
  if (c->d_p1 && c->d_p2) return SHARPY_OK;
  const int nd = c->ev.n_det;
  const int64_t K = c->ev.n_bins;
  if ((int64_t)c->h_wamp2.size() != nd * K || (int64_t)c->h_basis.size() != kNBasis * K) return SHARPY_ESTATE;
  std::vector<double> p1((size_t)nd * kNBasis * K), p2((size_t)nd * kNPair * K);
  auto prefix = [&](double* out, auto term) {
    double s = 0.0, cmp = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      const double t = term(k);
      const double u = s + t;
      cmp += std::fabs(s) >= std::fabs(t) ? (s - u) + t : (t - u) + s;
      s = u;
      out[k] = s + cmp;
    }
  };
  for (int a = 0; a < nd; ++a) {
    const double* W = c->h_wamp2.data() + (size_t)a * K;
    for (int m = 0; m < kNBasis; ++m) {
      const double* Bm = c->h_basis.data() + (size_t)m * K;
      prefix(p1.data() + ((size_t)a * kNBasis + m) * K, [&](int64_t k) { return W[k] * Bm[k]; });
      for (int n2 = m; n2 < kNBasis; ++n2) {
        const double* Bn = c->h_basis.data() + (size_t)n2 * K;
        const int pi = m * kNBasis - m * (m - 1) / 2 + (n2 - m);
        prefix(p2.data() + ((size_t)a * kNPair + pi) * K, [&](int64_t k) { return W[k] * Bm[k] * Bn[k]; });
      }
    }
  }
  if (cudaMalloc(&c->d_p1, p1.size() * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_p2, p2.size() * sizeof(double)) != cudaSuccess) {
    cudaFree(c->d_p1);
    cudaFree(c->d_p2);
    c->d_p1 = c->d_p2 = nullptr;
    return SHARPY_ENOMEM;
  }
  if (cudaMemcpy(c->d_p1, p1.data(), p1.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_p2, p2.data(), p2.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return SHARPY_ECUDA;
  c->ev.p1 = c->d_p1;
  c->ev.p2 = c->d_p2;
  return SHARPY_OK;
}

int enqueue_local_metric(sharpy_ctx* c, int64_t n, const double* theta, const double* beta_ptr, double beta,
                         double* mass, double* minv, double* chol, cudaStream_t s) {
  if (c->model.model == SHARPY_MODEL_TAYLORF2) {
    const int rc = ensure_fisher_tables(c);
    if (rc) return rc;
  }
  local_metric_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(c->model, c->ev, n, theta, beta_ptr, beta, mass,
                                                                   minv, chol, c->d_status);
  SHARPY_CUDA_TRY(cudaGetLastError());
  return SHARPY_OK;
}

}  // namespace sharpy

extern "C" int sharpy_local_metric(sharpy_ctx* c, int64_t n, const double* theta, double beta, double* mass,
                                   double* inv_mass, double* chol, sharpy_stream stream) {
  int rc = check_ctx(c, true);
  if (rc) return rc;
  if (n < 1 || n > ((int64_t)1 << 31) || !theta || !(beta >= 0.0 && beta <= 1.0) || (!mass && !inv_mass && !chol))
    return SHARPY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return enqueue_local_metric(c, n, theta, nullptr, beta, mass, inv_mass, chol, s);
}
