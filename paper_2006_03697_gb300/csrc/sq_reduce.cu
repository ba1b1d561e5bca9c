// Fermi level and contraction kernels (FP64).
//
//   R^j      = sum_q rho_q^j                                    (node sums, fixed order)
//   F_k      = sum'_j cos(j theta_k) R^j,  theta_k = pi (k + 1/2) / M
//   N(mu)    = 2 sum'_j c^j(mu) R^j = (4/M) sum_k g((chi + zeta cos theta_k - mu)/kT) F_k
// because c^j = (2/M) sum_k g(cos theta_k) cos(j theta_k) is the M-point Chebyshev-Gauss
// rule for the Clenshaw-Curtis coefficient integral of Sec. 4; bisection on N(mu) = N_e.
// The contraction evaluates c^j, d^j (coefficients of r g(r), App. A) and s^j (entropy
// function) at mu and forms rho_q, E_band, E_s, E_nl and sigma (Sec. 4 stress sums).
#include <algorithm>
#include <cmath>

#include "sq_device.cuh"

namespace sq {

// g ln g + (1 - g) ln(1 - g) at g = fermi(x), stable form -[ln(1+e^-|x|) + |x| e^-|x|/(1+e^-|x|)]
__device__ __forceinline__ double entropy_d(double x) {
  const double ax = fabs(x), ex = exp(-ax);
  return -(log1p(ex) + ax * ex / (1.0 + ex));
}

__global__ void k_rsum(const double* __restrict__ mom, int Nd, int n_pl, double* __restrict__ R) {
  __shared__ double sh[256];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int q = threadIdx.x; q < Nd; q += blockDim.x) s += mom[((size_t)q * (n_pl + 1) + j) * SQ_N_MOMENTS];
  s = block_sum_d(s, sh);
  if (threadIdx.x == 0) R[j] = s;
}

__global__ void k_cosF(const double* __restrict__ R, int n_pl, int M, double* __restrict__ F) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const double th = M_PI * (k + 0.5) / M;
  double s = 0.5 * R[0];
  for (int j = 1; j <= n_pl; ++j) s += cos(j * th) * R[j];
  F[k] = s;
}

// Single block. scal[0], scal[1]: bounds; writes scal[2] = mu, status[kStNoBracket].
__global__ void k_bisect(const double* __restrict__ F, int M, double kT, double n_e, double* __restrict__ scal,
                         int* __restrict__ status) {
  __shared__ double sh[1024];
  double mu = 0.0;
  const bool ok = fermi_bisect_rule(F, M, scal[0], scal[1], kT, n_e, sh, &mu);
  if (threadIdx.x == 0) {
    scal[2] = ok ? mu : NAN;
    status[kStNoBracket] = ok ? 0 : 1;
  }
}

// Coefficients at mu = scal[3]: block 0 -> c, 1 -> d (r g(r)), 2 -> s (entropy function).
__global__ void k_coef(const double* __restrict__ scal, double kT, int n_pl, int M, double* __restrict__ coef) {
  extern __shared__ double fv[];
  const double lam_lo = scal[0], lam_hi = scal[1], mu = scal[3];
  const double chi_q = 0.5 * (lam_hi + lam_lo), zeta_q = 0.5 * (lam_hi - lam_lo);
  const int which = blockIdx.x;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const double r = cos(M_PI * (k + 0.5) / M);
    const double x = (chi_q + zeta_q * r - mu) / kT;
    fv[k] = (which == 0) ? fermi_occ(x) : (which == 1) ? r * fermi_occ(x) : entropy_d(x);
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= n_pl; j += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < M; ++k) s += fv[k] * cos(j * (M_PI * (k + 0.5) / M));
    coef[which * (n_pl + 1) + j] = 2.0 / M * s;
  }
}

constexpr int kNPart = 20;

__global__ void k_contract(const double* __restrict__ mom, const double* __restrict__ coef,
                           const double* __restrict__ scal, const double* __restrict__ v, int Nd, int n_pl,
                           double dV, double* __restrict__ rho, double* __restrict__ part) {
  __shared__ double sh[256];
  const double lam_lo = scal[0], lam_hi = scal[1];
  const double chi_q = 0.5 * (lam_hi + lam_lo), zeta_q = 0.5 * (lam_hi - lam_lo);
  const double* c = coef;
  const double* d = coef + (n_pl + 1);
  const double* s = coef + 2 * (n_pl + 1);
  double acc[kNPart];
  for (int k = 0; k < kNPart; ++k) acc[k] = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Nd; q += gridDim.x * blockDim.x) {
    double r = 0.0;
    double loc[kNPart];
    for (int k = 0; k < kNPart; ++k) loc[k] = 0.0;
    for (int j = 0; j <= n_pl; ++j) {
      const double wp = (j == 0) ? 0.5 : 1.0;
      const double* m = mom + ((size_t)q * (n_pl + 1) + j) * SQ_N_MOMENTS;
      const double cj = wp * c[j];
      r += cj * m[0];
      loc[0] += wp * (chi_q * c[j] + zeta_q * d[j]) * m[0];
      loc[1] += wp * s[j] * m[0];
      loc[2] += cj * m[7];
      for (int k = 0; k < 6; ++k) loc[3 + k] += cj * m[1 + k];
      for (int k = 0; k < 9; ++k) loc[9 + k] += cj * m[8 + k];
    }
    rho[q] = 2.0 / dV * r;
    loc[18] = r;
    loc[19] = v[q] * r;   // |dOmega| V_q rho_q / 2
    for (int k = 0; k < kNPart; ++k) acc[k] += loc[k];
  }
  for (int k = 0; k < kNPart; ++k) {
    const double v = block_sum_d(acc[k], sh);
    if (threadIdx.x == 0) part[blockIdx.x * kNPart + k] = v;
  }
}

// out (scal + 16): [E_band, E_s, E_nl, N_check, sigma(9, row-major), E_pot, P]
// E_pot = |dOmega| sum_q V_q rho_q; P = the App. A pressure restricted to the kinetic and
// nonlocal terms: -(1/(3|Omega|)) [-2 (E_band - E_pot) - E_nl - 4 sum_q sum' c^j tr S^j_q]
// (the V_eff part of -4 tr(D H) goes with the exchange-correlation / electrostatic terms)
__global__ void k_contract_final(const double* __restrict__ part, int nblk, double kT, double vol,
                                 double* __restrict__ scal) {
  if (threadIdx.x != 0) return;
  double tot[kNPart];
  for (int k = 0; k < kNPart; ++k) tot[k] = 0.0;
  for (int b = 0; b < nblk; ++b)
    for (int k = 0; k < kNPart; ++k) tot[k] += part[b * kNPart + k];
  double* out = scal + 16;
  out[0] = 2.0 * tot[0];
  out[1] = 2.0 * kT * tot[1];
  const double E_nl = 2.0 * tot[2];
  out[2] = E_nl;
  out[3] = 2.0 * tot[18];   // |dOmega| sum_q rho_q = 2 sum_q sum' c rho^j
  const int ka[6] = {0, 1, 2, 1, 0, 0}, kb[6] = {0, 1, 2, 2, 2, 1};
  double sig[9];
  for (int k = 0; k < 9; ++k) sig[k] = 0.0;
  for (int k = 0; k < 6; ++k) {
    sig[3 * ka[k] + kb[k]] += 2.0 * tot[3 + k];
    if (ka[k] != kb[k]) sig[3 * kb[k] + ka[k]] += 2.0 * tot[3 + k];
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      sig[3 * a + b] += -2.0 * ((a == b ? 0.5 * E_nl : 0.0) + 2.0 * tot[9 + 3 * a + b]);
  for (int k = 0; k < 9; ++k) out[4 + k] = sig[k] / vol;
  const double E_pot = 2.0 * tot[19];
  out[13] = E_pot;
  out[14] = -(-2.0 * (out[0] - E_pot) - E_nl - 4.0 * (tot[9] + tot[13] + tot[17])) / (3.0 * vol);
}

__global__ void k_set_scalar(double* __restrict__ scal, int idx, double v) { scal[idx] = v; }

// Bisection on the node sums already in d.R (the whole cell's, or the caller's allreduced ones)
static int fermi_from_R(sq_handle* h, double* mu_out) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  k_cosF<<<(h->M + 255) / 256, 256, 0, s>>>(h->d.R, g.n_pl, h->M, h->d.cosF);
  SQ_LAUNCH_CHECK(h);
  k_bisect<<<1, 1024, 0, s>>>(h->d.cosF, h->M, h->kT, h->n_e, h->d.scal, h->d.status);
  SQ_LAUNCH_CHECK(h);
  double mu = 0.0;
  int st[kStCount];
  SQ_CUDA_TRY(h, cudaMemcpyAsync(&mu, h->d.scal + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
  SQ_CUDA_TRY(h, cudaMemcpyAsync(st, h->d.status, sizeof(st), cudaMemcpyDeviceToHost, s));
  SQ_CUDA_TRY(h, cudaStreamSynchronize(s));
  if (st[kStBadBounds]) return fail(h, SQ_ERR_CUDA, "spectral bounds are not finite or empty");
  if (st[kStOverflow]) return fail(h, SQ_ERR_CUDA, "internal list capacity exceeded");
  if (st[kStNoBracket]) return fail(h, SQ_ERR_NO_BRACKET, "N(mu) - N_e has no sign change on the bisection bracket");
  if (mu_out) *mu_out = mu;
  return SQ_OK;
}

int run_fermi(sq_handle* h, double* mu_out) {
  k_rsum<<<h->geo.n_pl + 1, 256, 0, h->stream>>>(h->d.mom, h->Nd, h->geo.n_pl, h->d.R);
  SQ_LAUNCH_CHECK(h);
  return fermi_from_R(h, mu_out);
}

int run_node_sums(sq_handle* h, double* R_out) {
  cudaStream_t s = h->stream;
  k_rsum<<<h->geo.n_pl + 1, 256, 0, s>>>(h->d.mom, h->Nd, h->geo.n_pl, h->d.R);
  SQ_LAUNCH_CHECK(h);
  SQ_CUDA_TRY(h, cudaMemcpyAsync(R_out, h->d.R, sizeof(double) * (h->geo.n_pl + 1), cudaMemcpyDeviceToHost, s));
  SQ_CUDA_TRY(h, cudaStreamSynchronize(s));
  return SQ_OK;
}

int run_fermi_sums(sq_handle* h, const double* R_host, double* mu_out) {
  SQ_CUDA_TRY(h, cudaMemcpyAsync(h->d.R, R_host, sizeof(double) * (h->geo.n_pl + 1), cudaMemcpyHostToDevice,
                                 h->stream));
  return fermi_from_R(h, mu_out);
}

__global__ void k_copy_scalar(double* __restrict__ scal, int dst, int src) { scal[dst] = scal[src]; }

// The Fermi level and the contraction with nothing crossing to the host (graph capture): mu
// stays in scal[2] (NaN and the no-bracket status word when there is no sign change), the
// contraction takes it from there and leaves its outputs in scal[16 ..].
int run_fermi_contraction_device(sq_handle* h) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  k_rsum<<<g.n_pl + 1, 256, 0, s>>>(h->d.mom, h->Nd, g.n_pl, h->d.R);
  SQ_LAUNCH_CHECK(h);
  k_cosF<<<(h->M + 255) / 256, 256, 0, s>>>(h->d.R, g.n_pl, h->M, h->d.cosF);
  SQ_LAUNCH_CHECK(h);
  k_bisect<<<1, 1024, 0, s>>>(h->d.cosF, h->M, h->kT, h->n_e, h->d.scal, h->d.status);
  SQ_LAUNCH_CHECK(h);
  k_copy_scalar<<<1, 1, 0, s>>>(h->d.scal, 3, 2);
  SQ_LAUNCH_CHECK(h);
  k_coef<<<3, 256, sizeof(double) * h->M, s>>>(h->d.scal, h->kT, g.n_pl, h->M, h->d.coef);
  SQ_LAUNCH_CHECK(h);
  const int nblk = std::min(1024, (h->Nd + 255) / 256);
  k_contract<<<nblk, 256, 0, s>>>(h->d.mom, h->d.coef, h->d.scal, h->d.v64, h->Nd, g.n_pl, g.dV, h->d.rho, h->d.part);
  SQ_LAUNCH_CHECK(h);
  k_contract_final<<<1, 32, 0, s>>>(h->d.part, nblk, h->kT, h->vol, h->d.scal);
  SQ_LAUNCH_CHECK(h);
  return SQ_OK;
}

int run_contraction(sq_handle* h, double mu, double* rho_dev, double* out_host) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  k_set_scalar<<<1, 1, 0, s>>>(h->d.scal, 3, mu);
  SQ_LAUNCH_CHECK(h);
  k_coef<<<3, 256, sizeof(double) * h->M, s>>>(h->d.scal, h->kT, g.n_pl, h->M, h->d.coef);
  SQ_LAUNCH_CHECK(h);
  const int nblk = std::min(1024, (h->Nd + 255) / 256);
  k_contract<<<nblk, 256, 0, s>>>(h->d.mom, h->d.coef, h->d.scal, h->d.v64, h->Nd, g.n_pl, g.dV, rho_dev, h->d.part);
  SQ_LAUNCH_CHECK(h);
  k_contract_final<<<1, 32, 0, s>>>(h->d.part, nblk, h->kT, h->vol, h->d.scal);
  SQ_LAUNCH_CHECK(h);
  if (out_host) {
    SQ_CUDA_TRY(h, cudaMemcpyAsync(out_host, h->d.scal + 16, 15 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SQ_CUDA_TRY(h, cudaStreamSynchronize(s));
  }
  return SQ_OK;
}


// ---------------------------------------------------------------- per-node bounds mode
// Every node q has its own interval (chi_q, zeta_q) and so its own coefficients
// c_q^j(mu) = (2/M) sum_k g((chi_q + zeta_q cos theta_k - mu)/kT) cos(j theta_k), and
//   N(mu) = 2 sum_q sum'_j c_q^j rho_q^j = (4/M) sum_q sum_k g(...) F_q(k),
//   F_q(k) = sum'_j cos(j theta_k) rho_q^j      (one table of N_d x M, formed once per search).
// tab[t] = cos(pi t / (2 M)), so cos(j theta_k) = tab[j (2 k + 1) mod 4 M].

__global__ void k_cosF_nodes(const double* __restrict__ mom, int Nd, int n_pl, int M, const double* __restrict__ tab,
                             double* __restrict__ F) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (k >= M || q >= Nd) return;
  const double* m = mom + (size_t)q * (n_pl + 1) * SQ_N_MOMENTS;
  const long long twoM4 = 4LL * M, odd = 2LL * k + 1;
  double s = 0.5 * m[0];
  for (int j = 1; j <= n_pl; ++j) s += tab[(j * odd) % twoM4] * m[(size_t)j * SQ_N_MOMENTS];
  F[(size_t)q * M + k] = s;
}

// part[block] = (4/M) sum over the block's nodes and all k of g((chi_q + zeta_q cos theta_k - mu)/kT) F_q(k)
__global__ void k_count_nodes(const double* __restrict__ F, const double* __restrict__ nbnd, int Nd, int M,
                              const double* __restrict__ tab, double kT, double mu, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int q = blockIdx.x; q < Nd; q += gridDim.x) {
    const double lo = nbnd[2 * q], hi = nbnd[2 * q + 1];
    const double chi_q = 0.5 * (hi + lo), zeta_q = 0.5 * (hi - lo);
    const double* Fq = F + (size_t)q * M;
    for (int k = threadIdx.x; k < M; k += blockDim.x)
      acc += fermi_occ((chi_q + zeta_q * tab[2 * k + 1] - mu) / kT) * Fq[k];
  }
  const double t = block_sum_d(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = 4.0 / M * t;
}

// out[0] = sum of part[0..n) in order; with ext: out[1] = min lo_q, out[2] = max hi_q
__global__ void k_sum_parts(const double* __restrict__ part, int n, const double* __restrict__ nbnd, int Nd,
                            double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < n; ++i) t += part[i];
  out[0] = t;
  if (nbnd) {
    double lo = INFINITY, hi = -INFINITY;
    for (int q = 0; q < Nd; ++q) {
      lo = fmin(lo, nbnd[2 * q]);
      hi = fmax(hi, nbnd[2 * q + 1]);
    }
    out[1] = lo;
    out[2] = hi;
  }
}

constexpr int kCountBlocks = 1024;

int run_fermi_nodes(sq_handle* h, double* mu_out) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  const int M = h->M;
  k_cosF_nodes<<<dim3((M + 255) / 256, h->Nd), 256, 0, s>>>(h->d.mom, h->Nd, g.n_pl, M, h->d.costab, h->d.nF);
  SQ_LAUNCH_CHECK(h);
  double* out = h->d.scal + 40;   // [count, min lo, max hi]
  auto count = [&](double mu, double* res, bool ext) -> int {
    k_count_nodes<<<kCountBlocks, 256, 0, s>>>(h->d.nF, h->d.nbnd, h->Nd, M, h->d.costab, h->kT, mu, h->d.npart);
    SQ_LAUNCH_CHECK(h);
    k_sum_parts<<<1, 32, 0, s>>>(h->d.npart, kCountBlocks, ext ? h->d.nbnd : nullptr, h->Nd, out);
    SQ_LAUNCH_CHECK(h);
    SQ_CUDA_TRY(h, cudaMemcpyAsync(res, out, (ext ? 3 : 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    SQ_CUDA_TRY(h, cudaStreamSynchronize(s));
    return SQ_OK;
  };
  // the shared mode's rule on [min lo_q - 40 kT, max hi_q + 40 kT]
  double e[3];
  int rc = count(0.0, e, true);
  if (rc != SQ_OK) return rc;
  double lo = e[1] - 40.0 * h->kT, hi = e[2] + 40.0 * h->kT, nlo = 0.0, nhi = 0.0;
  if ((rc = count(lo, &nlo, false)) != SQ_OK || (rc = count(hi, &nhi, false)) != SQ_OK) return rc;
  if (!(nlo < h->n_e && h->n_e < nhi))
    return fail(h, SQ_ERR_NO_BRACKET, "N(mu) - N_e has no sign change on the bisection bracket");
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    double nm = 0.0;
    if ((rc = count(mid, &nm, false)) != SQ_OK) return rc;
    if (nm < h->n_e) lo = mid;
    else hi = mid;
    if (hi - lo < 1e-13 * std::max(1.0, std::fabs(mid))) break;
  }
  if (mu_out) *mu_out = 0.5 * (lo + hi);
  return SQ_OK;
}

// One block per node: its coefficients c, d, s at mu (M-point Chebyshev-Gauss rule, as k_coef)
// and its contraction terms (the per-node rows of k_contract's partial sums), rho_q.
__global__ void k_contract_nodes(const double* __restrict__ mom, const double* __restrict__ nbnd,
                                 const double* __restrict__ v, int Nd, int n_pl, int M, const double* __restrict__ tab,
                                 double kT, double mu, double dV, double* __restrict__ rho, double* __restrict__ rows) {
  extern __shared__ double sm[];
  double* fv = sm;                       // [3][M]
  double* cf = sm + 3 * (size_t)M;       // [3][n_pl + 1]
  const int q = blockIdx.x;
  const double lo = nbnd[2 * q], hi = nbnd[2 * q + 1];
  const double chi_q = 0.5 * (hi + lo), zeta_q = 0.5 * (hi - lo);
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const double r = tab[2 * k + 1];
    const double x = (chi_q + zeta_q * r - mu) / kT;
    const double gx = fermi_occ(x);
    const double ax = fabs(x), ex = exp(-ax);
    fv[k] = gx;
    fv[M + k] = r * gx;
    fv[2 * M + k] = -(log1p(ex) + ax * ex / (1.0 + ex));
  }
  __syncthreads();
  const long long twoM4 = 4LL * M;
  for (int t = threadIdx.x; t < 3 * (n_pl + 1); t += blockDim.x) {
    const int which = t / (n_pl + 1), j = t % (n_pl + 1);
    const double* f = fv + (size_t)which * M;
    double acc = 0.0;
    for (int k = 0; k < M; ++k) acc += f[k] * tab[((long long)j * (2 * k + 1)) % twoM4];
    cf[t] = 2.0 / M * acc;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double* c = cf;
  const double* d = cf + (n_pl + 1);
  const double* sc = cf + 2 * (n_pl + 1);
  double loc[kNPart];
  for (int k = 0; k < kNPart; ++k) loc[k] = 0.0;
  double r = 0.0;
  for (int j = 0; j <= n_pl; ++j) {
    const double wp = (j == 0) ? 0.5 : 1.0;
    const double* m = mom + ((size_t)q * (n_pl + 1) + j) * SQ_N_MOMENTS;
    const double cj = wp * c[j];
    r += cj * m[0];
    loc[0] += wp * (chi_q * c[j] + zeta_q * d[j]) * m[0];
    loc[1] += wp * sc[j] * m[0];
    loc[2] += cj * m[7];
    for (int k = 0; k < 6; ++k) loc[3 + k] += cj * m[1 + k];
    for (int k = 0; k < 9; ++k) loc[9 + k] += cj * m[8 + k];
  }
  if (rho) rho[q] = 2.0 / dV * r;
  loc[18] = r;
  loc[19] = v[q] * r;
  for (int k = 0; k < kNPart; ++k) rows[(size_t)q * kNPart + k] = loc[k];
}

int run_contraction_nodes(sq_handle* h, double mu, double* rho_dev, double* out_host) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  const size_t smem = sizeof(double) * (3 * size_t(h->M) + 3 * size_t(g.n_pl + 1));
  SQ_CUDA_TRY(h, cudaFuncSetAttribute(k_contract_nodes, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  k_contract_nodes<<<h->Nd, 256, smem, s>>>(h->d.mom, h->d.nbnd, h->d.v64, h->Nd, g.n_pl, h->M, h->d.costab, h->kT,
                                            mu, g.dV, rho_dev, h->d.nrow);
  SQ_LAUNCH_CHECK(h);
  k_contract_final<<<1, 32, 0, s>>>(h->d.nrow, h->Nd, h->kT, h->vol, h->d.scal);
  SQ_LAUNCH_CHECK(h);
  if (out_host) {
    SQ_CUDA_TRY(h, cudaMemcpyAsync(out_host, h->d.scal + 16, 15 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SQ_CUDA_TRY(h, cudaStreamSynchronize(s));
  }
  return SQ_OK;
}

}  // namespace sq
