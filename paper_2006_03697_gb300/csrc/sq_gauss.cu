// Gauss Spectral Quadrature of the electron density (the SQ variant used for the SCF density,
// Sec. 5). For node q: k-step Lanczos on H_q from e_q (the column engine of the spectral
// bounds, all node columns of a wave of tiles together), the eigenvalues theta_qi of its
// tridiagonal T_q and the squared first components w_qi of their eigenvectors (Golub-Welsch:
// implicit QL with Wilkinson shifts, rotating only the first row of the eigenvector matrix);
// then [f(H_q)]_qq ~ sum_i w_qi f(theta_qi), exact for polynomials of degree <= 2k - 1.
// rho_q = (2 / |dOmega|) sum_i w_qi g(theta_qi), the Fermi level solves
// 2 sum_q sum_i w_qi g(theta_qi) = N_e (bisection, the rule of the Clenshaw-Curtis path) and
// E_band = 2 sum_q sum_i w_qi theta_qi g(theta_qi).
#include <algorithm>
#include <cmath>
#include <vector>

#include "sq_device.cuh"

namespace sq {

constexpr int kGaussMaxK = 128;

// Per column: Gauss nodes and weights from (alpha, beta, keff); zero weights beyond keff.
__global__ void k_gauss_eig(int ncols, int k, const double* __restrict__ alpha, const double* __restrict__ beta,
                            const int* __restrict__ keff, double* __restrict__ theta, double* __restrict__ wgt,
                            int* __restrict__ status) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncols) return;
  double d[kGaussMaxK], e[kGaussMaxK], z[kGaussMaxK];
  const int n = max(0, min(keff[col], k));
  for (int i = 0; i < n; ++i) {
    d[i] = alpha[(size_t)col * k + i];
    e[i] = (i < n - 1) ? beta[(size_t)col * k + i] : 0.0;
    z[i] = (i == 0) ? 1.0 : 0.0;
  }
  // implicit QL with Wilkinson shifts on the symmetric tridiagonal (d, e); z is the first row
  // of the accumulated rotations, so z_i^2 is the weight of eigenvalue d_i. The iteration is
  // the published EISPACK routine imtql2 (Bowdler, Martin, Reinsch and Wilkinson, "The QR and
  // QL algorithms for symmetric matrices", Numer. Math. 11, 1968; EISPACK, public domain),
  // restricted as in Golub and Welsch, "Calculation of Gauss quadrature rules", Math. Comp. 23,
  // 1969: only the first row of the eigenvector matrix is rotated.
  bool ok = true;
  for (int l = 0; l < n && ok; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;
      for (; m < n - 1; ++m) {
        const double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) + dd == dd) break;   // e[m] below half an ulp of its diagonal neighbours
      }
      if (m == l) break;
      if (iter == 60) {
        ok = false;
        break;
      }
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      int i = m - 1;
      bool underflow = false;
      for (; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[m] = 0.0;
          underflow = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        const double zf = z[i + 1];
        z[i + 1] = s * z[i] + c * zf;
        z[i] = c * z[i] - s * zf;
      }
      if (underflow) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  if (!ok) atomicOr(status + kStNoConverge, 1);
  for (int i = 0; i < k; ++i) {
    theta[(size_t)col * k + i] = (i < n) ? d[i] : 0.0;
    wgt[(size_t)col * k + i] = (i < n && ok) ? z[i] * z[i] : 0.0;
  }
}

// part[block] = sum over the block's columns of 2 sum_i w g((theta - mu) / kT) (fixed order)
__global__ void k_gauss_count(int ncols, int k, const double* __restrict__ theta, const double* __restrict__ wgt,
                              double mu, double kT, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < ncols; col += gridDim.x * blockDim.x)
    for (int i = 0; i < k; ++i) {
      const double w = wgt[(size_t)col * k + i];
      if (w != 0.0) acc += 2.0 * w * fermi_occ((theta[(size_t)col * k + i] - mu) / kT);
    }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Smallest and largest Gauss node with a non-zero weight: per block, then (k_gauss_minmax_final)
// over the blocks; the Fermi bracket's ends, without copying the N_d k nodes to the host.
__global__ void k_gauss_minmax(int n, const double* __restrict__ theta, const double* __restrict__ wgt,
                               double* __restrict__ part) {
  __shared__ double slo[256], shi[256];
  double lo = INFINITY, hi = -INFINITY;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (wgt[i] != 0.0) {
      lo = fmin(lo, theta[i]);
      hi = fmax(hi, theta[i]);
    }
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + st]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + st]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = slo[0];
    part[2 * blockIdx.x + 1] = shi[0];
  }
}

__global__ void k_gauss_minmax_final(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double lo = INFINITY, hi = -INFINITY;
  for (int b = 0; b < nblk; ++b) {
    lo = fmin(lo, part[2 * b]);
    hi = fmax(hi, part[2 * b + 1]);
  }
  out[0] = lo;
  out[1] = hi;
}

// out[0] = sum of part[0..n) in order (one thread)
__global__ void k_gauss_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < n; ++i) t += part[i];
  out[0] = t;
}

// rho at every valid node and the band-energy partial sums per block
__global__ void k_gauss_rho(Geo g, int ntiles_total, int k, const double* __restrict__ theta,
                            const double* __restrict__ wgt, double mu, double kT, double* __restrict__ rho,
                            double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  const int ncols = ntiles_total * g.B;
  for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < ncols; col += gridDim.x * blockDim.x) {
    const int t = col / g.B, q = col % g.B;
    int o[3], qo[3];
    tile_origin(g, t, o);
    node_offset(g, q, qo);
    if (!node_valid(g, o, qo)) continue;
    double r = 0.0, eb = 0.0;
    for (int i = 0; i < k; ++i) {
      const double w = wgt[(size_t)col * k + i];
      if (w == 0.0) continue;
      const double th = theta[(size_t)col * k + i];
      const double f = w * fermi_occ((th - mu) / kT);
      r += f;
      eb += f * th;
    }
    const int node = (o[0] + qo[0]) + g.n[0] * ((o[1] + qo[1]) + g.n[1] * (o[2] + qo[2]));
    rho[node] = 2.0 / g.dV * r;
    acc += 2.0 * eb;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

template <typename Real>
static int gauss_t(sq_handle* h, int k, double* mu_out, double* rho_host, double* e_band_out) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  // tiles per Lanczos wave: k + 2 vectors and the projections per tile under ~16 GiB, at most the
  // list capacity of a sweep wave
  const size_t per_tile = ((size_t)(k + 2) * g.Upts + (size_t)g.r_cap) * g.B * sizeof(Real) +
                          (size_t)g.B * (5 * k + 8) * sizeof(double);
  // at most 16 GiB, and at most 80 % of the free device memory, of Krylov waves
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = size_t(16) << 30;
  }
  const size_t fixed = 2 * sizeof(double) * (size_t)g.n_tiles * g.B * k + sizeof(double) * (size_t)h->Nd;
  const size_t wave_budget = std::min<size_t>(size_t(16) << 30, free_b > fixed ? (free_b - fixed) / 10 * 8 : 0);
  const int wt = int(std::max<size_t>(1, std::min<size_t>(wave_budget / per_tile, (size_t)h->wave_cap)));
  const int ncols_all = g.n_tiles * g.B;
  std::vector<void*> bufs;
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    bufs.push_back(*p);
    return true;
  };
  auto release = [&]() {
    for (void* p : bufs) cudaFree(p);
    bufs.clear();
  };
  Real *V = nullptr, *W = nullptr, *P = nullptr;
  double *C = nullptr, *theta = nullptr, *wgt = nullptr, *part = nullptr, *sum = nullptr, *rho = nullptr;
  const int nblk = 1024;
  if (!alloc((void**)&V, sizeof(Real) * (size_t)(k + 1) * wt * g.Upts * g.B) ||
      !alloc((void**)&W, sizeof(Real) * (size_t)wt * g.Upts * g.B) ||
      !alloc((void**)&P, sizeof(Real) * (size_t)wt * g.r_cap * g.B) ||
      !alloc((void**)&C, sizeof(double) * (size_t)wt * g.B * (5 * k + 8)) ||
      !alloc((void**)&theta, sizeof(double) * (size_t)ncols_all * k) ||
      !alloc((void**)&wgt, sizeof(double) * (size_t)ncols_all * k) ||
      !alloc((void**)&part, sizeof(double) * nblk) || !alloc((void**)&sum, 2 * sizeof(double)) ||
      !alloc((void**)&rho, sizeof(double) * h->Nd)) {
    release();
    return fail(h, SQ_ERR_OOM, "device allocation for the Gauss quadrature failed");
  }
  int rc = SQ_OK;
  if (cudaMemsetAsync(h->d.status, 0, sizeof(int) * kStCount, s) != cudaSuccess)
    rc = fail(h, SQ_ERR_CUDA, "status reset failed");
  for (int t0 = 0; t0 < g.n_tiles && rc == SQ_OK; t0 += wt) {
    const Wave w{t0, std::min(wt, g.n_tiles - t0), nullptr};
    rc = lanczos_columns<Real>(h, w, 1, k, V, W, P, C, &h->wb);
    if (rc != SQ_OK) break;
    const int ncols = w.ntiles * g.B;
    const double* alpha = C + (size_t)3 * ncols * (k + 1);
    const double* beta = alpha + (size_t)ncols * k;
    const int* keff = (const int*)(beta + (size_t)ncols * k);
    k_gauss_eig<<<(ncols + 63) / 64, 64, 0, s>>>(ncols, k, alpha, beta, keff, theta + (size_t)t0 * g.B * k,
                                                wgt + (size_t)t0 * g.B * k, h->d.status);
    if (cudaGetLastError() != cudaSuccess) rc = fail(h, SQ_ERR_CUDA, "k_gauss_eig launch failed");
  }
  // Fermi level: bisection with the Clenshaw-Curtis path's rule; the bracket from the extreme
  // weighted Gauss nodes (device reduction, two doubles to the host)
  double tmin = 0.0, tmax = 0.0;
  if (rc == SQ_OK) {
    const int mblk = std::min(nblk / 2, std::max(1, (ncols_all * k + 255) / 256));
    double ext[2];
    k_gauss_minmax<<<mblk, 256, 0, s>>>(ncols_all * k, theta, wgt, part);
    k_gauss_minmax_final<<<1, 32, 0, s>>>(part, mblk, sum);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(ext, sum, sizeof(ext), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = fail(h, SQ_ERR_CUDA, "Gauss node extremes failed");
    } else if (!(ext[0] <= ext[1])) {
      rc = fail(h, SQ_ERR_NO_BRACKET, "no Gauss node carries weight");
    } else {
      tmin = ext[0];
      tmax = ext[1];
    }
  }
  auto count = [&](double mu, double* out) -> int {
    k_gauss_count<<<nblk, 256, 0, s>>>(ncols_all, k, theta, wgt, mu, h->kT, part);
    k_gauss_sum<<<1, 32, 0, s>>>(part, nblk, sum);
    if (cudaGetLastError() != cudaSuccess) return SQ_ERR_CUDA;
    if (cudaMemcpyAsync(out, sum, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SQ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SQ_ERR_CUDA;
    return SQ_OK;
  };
  double mu = 0.0;
  if (rc == SQ_OK) {
    double lo = tmin - 40.0 * h->kT, hi = tmax + 40.0 * h->kT, nlo = 0.0, nhi = 0.0;
    if (count(lo, &nlo) != SQ_OK || count(hi, &nhi) != SQ_OK) {
      rc = fail(h, SQ_ERR_CUDA, "electron count failed");
    } else if (!(nlo < h->n_e && h->n_e < nhi)) {
      rc = fail(h, SQ_ERR_NO_BRACKET, "N(mu) - N_e has no sign change on the bisection bracket");
    } else {
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        double nm = 0.0;
        if (count(mid, &nm) != SQ_OK) {
          rc = fail(h, SQ_ERR_CUDA, "electron count failed");
          break;
        }
        if (nm < h->n_e) lo = mid;
        else hi = mid;
        if (hi - lo < 1e-13 * std::max(1.0, std::fabs(mid))) break;
      }
      mu = 0.5 * (lo + hi);
    }
  }
  if (rc == SQ_OK) {
    k_gauss_rho<<<nblk, 256, 0, s>>>(g, g.n_tiles, k, theta, wgt, mu, h->kT, rho, part);
    k_gauss_sum<<<1, 32, 0, s>>>(part, nblk, sum);
    double eb = 0.0;
    int st[kStCount];
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&eb, sum, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        (rho_host && cudaMemcpyAsync(rho_host, rho, sizeof(double) * h->Nd, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        cudaMemcpyAsync(st, h->d.status, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = fail(h, SQ_ERR_CUDA, "Gauss density contraction failed");
    } else if (st[kStNoConverge]) {
      rc = fail(h, SQ_ERR_CUDA, "tridiagonal eigensolver did not converge");
    } else if (st[kStOverflow]) {
      rc = fail(h, SQ_ERR_CUDA, "internal list capacity exceeded");
    } else {
      if (mu_out) *mu_out = mu;
      if (e_band_out) *e_band_out = eb;
    }
  }
  release();
  return rc;
}

}  // namespace sq

extern "C" int sq_gauss_density(sq_handle* h, int k, double* mu_out, double* rho_out, double* e_band_out) {
  if (!h) return SQ_ERR_INVALID_ARG;
  if (k < 1 || k > sq::kGaussMaxK || k + 1 > 136)
    return sq::fail(h, SQ_ERR_INVALID_ARG, "Gauss quadrature order k must be in 1..128");
  if (h->precision == SQ_MIXED) return sq::gauss_t<float>(h, k, mu_out, rho_out, e_band_out);
  return sq::gauss_t<double>(h, k, mu_out, rho_out, e_band_out);
}
