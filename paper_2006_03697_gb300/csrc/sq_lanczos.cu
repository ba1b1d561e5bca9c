// Spectral bounds for the Chebyshev scaling chi_q, zeta_q of Sec. 4 (FP64 for SQ_FP64; for
// SQ_MIXED the Krylov vectors and H_q applications are FP32, the Gram-Schmidt coefficients,
// tridiagonal and Ritz values FP64 - the bounds are widened by 1 % of the width anyway).
//
// The paper takes chi_q and zeta_q from the extreme eigenvalues of H_q and does not say how
// they are obtained. Here: k-step Lanczos on the nodal Hamiltonian H_q of every node of a few
// sample tiles (one Lanczos column per node, all columns advanced together with the tile
// kernels), full reorthogonalisation by classical Gram-Schmidt applied twice, Ritz extremes
// of the tridiagonal matrix widened by their residual norms, the interval over all columns,
// then widened by 1 % of its width on each side. One interval serves every node (every H_q
// is a principal submatrix of the infinite-crystal H, so a shared interval is valid for all
// of them when it contains the sampled spectra with margin).
#include <algorithm>
#include <cmath>
#include <vector>

#include "sq_device.cuh"

namespace sq {

constexpr int kTileLz = 8;              // nodes per tile (columns per tile)
constexpr int kMaxLanczosVecs = 136;    // Krylov vectors held (k + 1, k <= 128 + 7)
constexpr int kLzDotChunks = 32;        // most chunks a dot product of a small wave is split into

// Start vector of the column of node q: 1 + (hash(i, node) mod 1009) / 1009 on the window
// (i = window-local index, C order z, y, x), zero elsewhere; normalised afterwards.
template <typename Real>
__global__ void k_lz_init(Geo g, Wave w, Real* __restrict__ V0) {
  const size_t per_tile = (size_t)g.Upts * g.B;
  const size_t total = per_tile * w.ntiles;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int tl = int(idx / per_tile);
    const int r = int(idx % per_tile);
    const int q = r % g.B, pt = r / g.B;
    const int ux = pt % g.U[0], uy = (pt / g.U[0]) % g.U[1], uz = pt / (g.U[0] * g.U[1]);
    int o[3], qo[3];
    tile_origin(g, wave_tile(w, tl), o);
    node_offset(g, q, qo);
    double v = 0.0;
    if (node_valid(g, o, qo) && in_window(g, qo, ux, uy, uz)) {
      const int kx = ux - qo[0], ky = uy - qo[1], kz = uz - qo[2];
      const unsigned long long i = (unsigned long long)((kz * (2 * g.m[1] + 1) + ky) * (2 * g.m[0] + 1) + kx);
      const unsigned long long node =
          (unsigned long long)((o[0] + qo[0]) + g.n[0] * ((o[1] + qo[1]) + g.n[1] * (o[2] + qo[2])));
      const unsigned long long hsh = (i * 2654435761ull + node * 40503ull) & 0xFFFFFFFFull;
      v = 1.0 + double(hsh % 1009ull) / 1009.0;
    }
    V0[idx] = Real(v);
  }
}

// Start vector e_q: one at node q's own point of the union window, zero elsewhere (and an
// all-zero column for padding nodes, which the mark-empty pass then skips).
template <typename Real>
__global__ void k_lz_init_unit(Geo g, Wave w, Real* __restrict__ V0) {
  const size_t per_tile = (size_t)g.Upts * g.B;
  const size_t total = per_tile * w.ntiles;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int tl = int(idx / per_tile);
    const int r = int(idx % per_tile);
    const int q = r % g.B, pt = r / g.B;
    int o[3], qo[3];
    tile_origin(g, wave_tile(w, tl), o);
    node_offset(g, q, qo);
    const int cpt = ((qo[2] + g.m[2]) * g.U[1] + (qo[1] + g.m[1])) * g.U[0] + (qo[0] + g.m[0]);
    V0[idx] = (node_valid(g, o, qo) && pt == cpt) ? Real(1) : Real(0);
  }
}

// out[col * ld + i] = <V_i, x>_col for i < nvec (one block per (i, tile); fixed-order sums:
// per thread in the vectors' precision, across threads in FP64)
template <typename Real>
__global__ void k_lz_dots(Geo g, Wave w, const Real* __restrict__ V, int nvec, size_t vstride,
                          const Real* __restrict__ x, double* __restrict__ out, int ld) {
  const int i = blockIdx.x, tl = blockIdx.y;
  const size_t base = (size_t)tl * g.Upts * g.B;
  const Real* Vi = V + (size_t)i * vstride + base;
  const Real* xt = x + base;
  const int q = threadIdx.x % g.B;
  Real s = Real(0);
  for (int e = threadIdx.x; e < g.Upts * g.B; e += blockDim.x) s += Vi[e] * xt[e];
  __shared__ double red[kThreads];
  red[threadIdx.x] = double(s);
  __syncthreads();
  if (threadIdx.x < g.B) {
    double t = 0.0;
    for (int th = q; th < kThreads; th += g.B) t += red[th];
    out[((size_t)tl * g.B + q) * ld + i] = t;
  }
}

// The same products for waves of few tiles (the Lanczos sample tiles): block (i, tile, c) sums
// chunk c of the tile's vector pair into part[((tile * nvec + i) * nch + c) * B + node], and
// k_lz_dots_sum adds the nch chunks of every (tile, node, i) in order, so a product spreads over
// nch times more blocks and the result does not depend on scheduling.
template <typename Real>
__global__ void k_lz_dots_part(Geo g, Wave w, const Real* __restrict__ V, int nvec, size_t vstride,
                               const Real* __restrict__ x, double* __restrict__ part, int nch) {
  const int i = blockIdx.x, tl = blockIdx.y, c = blockIdx.z;
  const size_t n = (size_t)g.Upts * g.B;
  const size_t len = ((n + nch - 1) / nch + g.B - 1) / g.B * g.B;   // chunks start at a node-0 slot
  const size_t e0 = (size_t)c * len, e1 = min(n, e0 + len);
  const size_t base = (size_t)tl * n;
  const Real* Vi = V + (size_t)i * vstride + base;
  const Real* xt = x + base;
  const int q = threadIdx.x % g.B;
  Real s = Real(0);
  for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) s += Vi[e] * xt[e];
  __shared__ double red[kThreads];
  red[threadIdx.x] = double(s);
  __syncthreads();
  if (threadIdx.x < g.B) {
    double t = 0.0;
    for (int th = q; th < kThreads; th += g.B) t += red[th];
    part[(((size_t)tl * nvec + i) * nch + c) * g.B + q] = t;
  }
}

__global__ void k_lz_dots_sum(const double* __restrict__ part, int ntiles, int nvec, int nch, int B,
                              double* __restrict__ out, int ld) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ntiles * nvec * B) return;
  const int q = k % B, i = (k / B) % nvec, tl = k / (B * nvec);
  double t = 0.0;
  for (int c = 0; c < nch; ++c) t += part[(((size_t)tl * nvec + i) * nch + c) * B + q];
  out[((size_t)tl * B + q) * ld + i] = t;
}

// out[(tile node) * ld + i] = V_i . x per node column, one launch (or two for few tiles)
template <typename Real>
static int lz_dots(sq_handle* h, const Wave& w, const Real* V, int nvec, size_t vstride, const Real* x, double* out,
                   int ld) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  const int blocks = nvec * w.ntiles;
  const int nch = std::max(1, std::min(kLzDotChunks, (2 * 152 + blocks - 1) / std::max(1, blocks)));
  if (blocks >= 2 * 152 || !h->d.lzdot || size_t(blocks) * nch * g.B > kLzDotCap) {
    k_lz_dots<Real><<<dim3(nvec, w.ntiles), kThreads, 0, s>>>(g, w, V, nvec, vstride, x, out, ld);
    SQ_LAUNCH_CHECK(h);
    return SQ_OK;
  }
  k_lz_dots_part<Real><<<dim3(nvec, w.ntiles, nch), kThreads, 0, s>>>(g, w, V, nvec, vstride, x, h->d.lzdot, nch);
  SQ_LAUNCH_CHECK(h);
  const int nk = w.ntiles * nvec * g.B;
  k_lz_dots_sum<<<(nk + 255) / 256, 256, 0, s>>>(h->d.lzdot, w.ntiles, nvec, nch, g.B, out, ld);
  SQ_LAUNCH_CHECK(h);
  return SQ_OK;
}

// x -= sum_i coef[col * ld + i] V_i; grid (blocks per tile, tiles): a block's coefficients
// (8 columns x nvec) are converted to the vectors' precision once, in shared memory
template <typename Real>
__global__ void k_lz_update(Geo g, Wave w, const Real* __restrict__ V, int nvec, size_t vstride,
                            const double* __restrict__ coef, int ld, Real* __restrict__ x) {
  __shared__ Real cf[kTileLz][kMaxLanczosVecs];
  const int tl = blockIdx.y;
  for (int k2 = threadIdx.x; k2 < g.B * nvec; k2 += blockDim.x) {
    const int q = k2 / nvec, i = k2 % nvec;
    cf[q][i] = Real(coef[((size_t)tl * g.B + q) * ld + i]);
  }
  __syncthreads();
  const size_t per_tile = (size_t)g.Upts * g.B;
  const size_t base = per_tile * tl;
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < per_tile; r += (size_t)gridDim.x * blockDim.x) {
    const int q = int(r % g.B);
    Real acc = Real(0);
    for (int i = 0; i < nvec; ++i) acc += cf[q][i] * V[(size_t)i * vstride + base + r];
    x[base + r] -= acc;
  }
}

// Per column: alpha_i = cA_i + cB_i, beta_i = ||w||; a column whose beta falls below
// 1e-12 max(1, |alpha_i|) stops with k_eff = i + 1 (keff < 0 while running).
__global__ void k_lz_step(int ncols, int i, int kk, int k, const double* __restrict__ cA, const double* __restrict__ cB,
                          int ld, const double* __restrict__ nrm, double* __restrict__ alpha, double* __restrict__ beta,
                          int* __restrict__ keff) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncols || keff[col] >= 0) return;
  const double a = cA[(size_t)col * ld + i] + cB[(size_t)col * ld + i];
  const double b = sqrt(nrm[(size_t)col * ld]);
  alpha[(size_t)col * k + i] = a;
  beta[(size_t)col * k + i] = b;
  if (i == kk - 1 || b <= 1e-12 * fmax(1.0, fabs(a))) keff[col] = i + 1;
}

// V_next = x / beta for running columns (zero otherwise). With first != 0: normalise the
// start vector in place (beta = sqrt(nrm)); a zero start vector marks an empty column.
template <typename Real>
__global__ void k_lz_scale(Geo g, Wave w, const Real* __restrict__ x, const double* __restrict__ nrm, int ld,
                           int* __restrict__ keff, Real* __restrict__ Vn, int first) {
  const size_t per_tile = (size_t)g.Upts * g.B;
  const size_t total = per_tile * w.ntiles;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int tl = int(idx / per_tile);
    const int q = int(idx % per_tile) % g.B;
    const size_t col = (size_t)tl * g.B + q;
    const double b = sqrt(nrm[col * ld]);
    const bool run = first ? (b > 0.0) : (keff[col] < 0);
    Vn[idx] = run ? Real(double(x[idx]) / b) : Real(0);
  }
}

__global__ void k_lz_mark_empty(int ncols, const double* __restrict__ nrm, int ld, int* __restrict__ keff) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col < ncols) keff[col] = (nrm[(size_t)col * ld] > 0.0) ? -1 : 0;
}

// Sturm count of eigenvalues of the tridiagonal (a, b) below x.
__device__ int sturm_count(const double* a, const double* b, int n, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < n; ++i) {
    d = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// |last component| of the unit eigenvector for the extreme eigenvalue theta, by two steps
// of inverse iteration with the shift just outside the spectrum (definite, so the
// unpivoted tridiagonal solve is stable).
__device__ double last_component(const double* a, const double* b, int n, double shift, double* y, double* dd) {
  for (int i = 0; i < n; ++i) y[i] = 1.0;
  for (int it = 0; it < 3; ++it) {
    // LDL^T of (T - shift I), then solve
    dd[0] = a[0] - shift;
    for (int i = 1; i < n; ++i) dd[i] = a[i] - shift - b[i - 1] * b[i - 1] / dd[i - 1];
    for (int i = 1; i < n; ++i) y[i] -= b[i - 1] / dd[i - 1] * y[i - 1];
    y[n - 1] /= dd[n - 1];
    for (int i = n - 2; i >= 0; --i) y[i] = (y[i] - b[i] * y[i + 1]) / dd[i];
    double nr = 0.0;
    for (int i = 0; i < n; ++i) nr += y[i] * y[i];
    nr = sqrt(nr);
    for (int i = 0; i < n; ++i) y[i] /= nr;
  }
  return fabs(y[n - 1]);
}

constexpr int kMaxLanczos = 128;

// One block: Ritz extremes with residual bounds per column, min / max over columns,
// widening by 1 % of the width; writes scal[8] = lo, scal[9] = hi.
__global__ void k_lz_bounds(int ncols, int k, const double* __restrict__ alpha, const double* __restrict__ beta,
                            const int* __restrict__ keff, double* __restrict__ scal) {
  __shared__ double slo[256], shi[256];
  double lo = INFINITY, hi = -INFINITY;
  double y[kMaxLanczos], dd[kMaxLanczos];
  for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
    const int n = keff[col];
    if (n <= 0) continue;
    const double* a = alpha + (size_t)col * k;
    const double* b = beta + (size_t)col * k;
    double gl = INFINITY, gu = -INFINITY;
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < n - 1 ? fabs(b[i]) : 0.0);
      gl = fmin(gl, a[i] - r);
      gu = fmax(gu, a[i] + r);
    }
    double l = gl, u = gu;                      // smallest eigenvalue: count(x) >= 1
    for (int it = 0; it < 200 && u - l > 1e-15 * fmax(1.0, fmax(fabs(l), fabs(u))); ++it) {
      const double mid = 0.5 * (l + u);
      if (sturm_count(a, b, n, mid) >= 1) u = mid; else l = mid;
    }
    const double tmin = 0.5 * (l + u);
    l = gl; u = gu;                             // largest eigenvalue: count(x) == n
    for (int it = 0; it < 200 && u - l > 1e-15 * fmax(1.0, fmax(fabs(l), fabs(u))); ++it) {
      const double mid = 0.5 * (l + u);
      if (sturm_count(a, b, n, mid) >= n) u = mid; else l = mid;
    }
    const double tmax = 0.5 * (l + u);
    const double bl = fabs(b[n - 1]);
    const double del = 1e-10 * fmax(gu - gl, 1e-300);
    const double rmin = (n > 1) ? bl * last_component(a, b, n, tmin - del, y, dd) : bl;
    const double rmax = (n > 1) ? bl * last_component(a, b, n, tmax + del, y, dd) : bl;
    lo = fmin(lo, tmin - rmin);
    hi = fmax(hi, tmax + rmax);
  }
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + s]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double wdt = shi[0] - slo[0];
    scal[8] = slo[0] - 0.01 * wdt;
    scal[9] = shi[0] + 0.01 * wdt;
  }
}

// The per-node bounds mode: each column's own interval (Ritz extremes widened by their residual
// norms, then by 1 % of that column's width, as the shared interval is formed from all sample
// columns) and the step coefficients the recurrence of that node uses, with the scaling rules
// of set_bounds (SQ_MIXED: FP32-exact 2 / zeta and -2 chi / zeta; the diagonal coefficient
// rounded once; the stencil's constant-mode offset and that rounding folded into the centre).
__global__ void k_lz_node_bounds(Geo g, Wave w, int k, const double* __restrict__ alpha, const double* __restrict__ beta,
                                 const int* __restrict__ keff, int mixed, double lap_offset, double* __restrict__ nbnd,
                                 double* __restrict__ ncoef) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= w.ntiles * g.B) return;
  int o[3], qo[3];
  tile_origin(g, wave_tile(w, col / g.B), o);
  node_offset(g, col % g.B, qo);
  if (!node_valid(g, o, qo)) return;
  const int node = (o[0] + qo[0]) + g.n[0] * ((o[1] + qo[1]) + g.n[1] * (o[2] + qo[2]));
  const int n = keff[col];
  if (n <= 0) return;
  double y[kMaxLanczos], dd[kMaxLanczos];
  const double* a = alpha + (size_t)col * k;
  const double* b = beta + (size_t)col * k;
  double gl = INFINITY, gu = -INFINITY;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < n - 1 ? fabs(b[i]) : 0.0);
    gl = fmin(gl, a[i] - r);
    gu = fmax(gu, a[i] + r);
  }
  double l = gl, u = gu;
  for (int it = 0; it < 200 && u - l > 1e-15 * fmax(1.0, fmax(fabs(l), fabs(u))); ++it) {
    const double mid = 0.5 * (l + u);
    if (sturm_count(a, b, n, mid) >= 1) u = mid; else l = mid;
  }
  const double tmin = 0.5 * (l + u);
  l = gl;
  u = gu;
  for (int it = 0; it < 200 && u - l > 1e-15 * fmax(1.0, fmax(fabs(l), fabs(u))); ++it) {
    const double mid = 0.5 * (l + u);
    if (sturm_count(a, b, n, mid) >= n) u = mid; else l = mid;
  }
  const double tmax = 0.5 * (l + u);
  const double bl = fabs(b[n - 1]);
  const double del = 1e-10 * fmax(gu - gl, 1e-300);
  const double rmin = (n > 1) ? bl * last_component(a, b, n, tmin - del, y, dd) : bl;
  const double rmax = (n > 1) ? bl * last_component(a, b, n, tmax + del, y, dd) : bl;
  double lo = tmin - rmin, hi = tmax + rmax;
  const double wdt = hi - lo;
  lo -= 0.01 * wdt;
  hi += 0.01 * wdt;
  // scaling of this node's recurrence (set_bounds, per node)
  double chi = 0.5 * (hi + lo), zeta = 0.5 * (hi - lo);
  double ca = 2.0 / zeta, cb = -2.0 * chi / zeta;
  if (mixed) {
    ca = double(float(ca));
    zeta = 2.0 / ca;
    cb = double(float(-2.0 * chi / zeta));
    chi = -cb * zeta / 2.0;
  }
  double cd = ca * g.lap0 + cb;
  if (mixed) cd = double(float(cd));
  const double eps = cd - (ca * g.lap0 + cb);
  chi -= lap_offset + eps / ca;
  nbnd[2 * node] = chi - zeta;
  nbnd[2 * node + 1] = chi + zeta;
  ncoef[2 * node] = ca;
  ncoef[2 * node + 1] = cd;
}

// k-step Lanczos (CGS2 reorthogonalisation) of every node column of the wave's tiles, from the
// hash start vector (start = 0, the spectral bounds) or from e_q (start = 1, Gauss SQ). V holds
// k + 1 vectors of the wave, W one, P the projections; C is (5 k + 8) doubles per column:
// cA, cB, nrm [ncols][k + 1], alpha, beta [ncols][k], keff (ints) - see lz_alpha etc.
template <typename Real>
int lanczos_columns(sq_handle* h, const Wave& w, int start, int k, Real* V, Real* W, Real* P, double* C,
                    WaveBufs* b) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  const int nst = w.ntiles;
  // never more steps than the region has dimensions (the Krylov space is exhausted)
  const long long nc = (long long)(2 * g.m[0] + 1) * (2 * g.m[1] + 1) * (2 * g.m[2] + 1);
  const int kk = int(std::min<long long>(k, nc));
  const int ncols = nst * g.B;
  const int ld = k + 1;
  const size_t vstride = (size_t)nst * g.Upts * g.B;
  double* cA = C;
  double* cB = cA + (size_t)ncols * ld;
  double* nrm = cB + (size_t)ncols * ld;
  double* alpha = nrm + (size_t)ncols * ld;
  double* beta = alpha + (size_t)ncols * k;
  int* keff = (int*)(beta + (size_t)ncols * k);
  const int eb = 1024;
  const int ub = int(std::min<size_t>(64, ((size_t)g.Upts * g.B + 255) / 256));   // update blocks per tile
  const int cb = (ncols + 127) / 128;
  // the sample tiles' lists (their own buffers) only change with the atoms; a graph capture
  // records the build
  int rc = SQ_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SQ_CUDA_TRY(h, cudaStreamIsCapturing(s, &cap));
  if (b != &h->lzb || !h->keep_lists || h->lz_lists_epoch != h->atoms_epoch || cap != cudaStreamCaptureStatusNone) {
    rc = build_wave_entries(h, w, b);
    if (rc != SQ_OK) return rc;
    if (b == &h->lzb) h->lz_lists_epoch = h->atoms_epoch;
  }
  if (start == 0) k_lz_init<Real><<<eb, 256, 0, s>>>(g, w, V);
  else k_lz_init_unit<Real><<<eb, 256, 0, s>>>(g, w, V);
  SQ_LAUNCH_CHECK(h);
  rc = lz_dots<Real>(h, w, V, 1, vstride, V, nrm, ld);
  if (rc != SQ_OK) return rc;
  k_lz_mark_empty<<<cb, 128, 0, s>>>(ncols, nrm, ld, keff);
  SQ_LAUNCH_CHECK(h);
  k_lz_scale<Real><<<eb, 256, 0, s>>>(g, w, V, nrm, ld, keff, V, 1);
  SQ_LAUNCH_CHECK(h);
  for (int i = 0; i < kk; ++i) {
    Real* Vi = V + (size_t)i * vstride;
    rc = launch_apply_h(h, w, Vi, W, P, *b);
    if (rc != SQ_OK) return rc;
    rc = lz_dots<Real>(h, w, V, i + 1, vstride, W, cA, ld);
    if (rc != SQ_OK) return rc;
    k_lz_update<Real><<<dim3(ub, nst), 256, 0, s>>>(g, w, V, i + 1, vstride, cA, ld, W);
    SQ_LAUNCH_CHECK(h);
    rc = lz_dots<Real>(h, w, V, i + 1, vstride, W, cB, ld);
    if (rc != SQ_OK) return rc;
    k_lz_update<Real><<<dim3(ub, nst), 256, 0, s>>>(g, w, V, i + 1, vstride, cB, ld, W);
    SQ_LAUNCH_CHECK(h);
    rc = lz_dots<Real>(h, w, W, 1, vstride, W, nrm, ld);
    if (rc != SQ_OK) return rc;
    k_lz_step<<<cb, 128, 0, s>>>(ncols, i, kk, k, cA, cB, ld, nrm, alpha, beta, keff);
    SQ_LAUNCH_CHECK(h);
    if (i < kk - 1) {
      k_lz_scale<Real><<<eb, 256, 0, s>>>(g, w, W, nrm, ld, keff, V + (size_t)(i + 1) * vstride, 0);
      SQ_LAUNCH_CHECK(h);
    }
  }
  return SQ_OK;
}

template int lanczos_columns<float>(sq_handle*, const Wave&, int, int, float*, float*, float*, double*, WaveBufs*);
template int lanczos_columns<double>(sq_handle*, const Wave&, int, int, double*, double*, double*, double*, WaveBufs*);

template <typename Real>
static int run_lanczos_t(sq_handle* h) {
  const int nst = int(h->lanczos_tiles.size());
  const int k = h->lanczos_k;
  const int ncols = nst * h->geo.B;
  const Wave w{0, nst, h->d.lz_tiles};
  // the sample tiles' lists go to their own buffers, so the sweep's lists (and W) stay valid
  int rc = lanczos_columns<Real>(h, w, 0, k, reinterpret_cast<Real*>(h->d.lzV), reinterpret_cast<Real*>(h->d.lzW),
                                 reinterpret_cast<Real*>(h->d.lzP), h->d.lzC, &h->lzb);
  if (rc != SQ_OK) return rc;
  const double* alpha = h->d.lzC + (size_t)3 * ncols * (k + 1);
  const double* beta = alpha + (size_t)ncols * k;
  const int* keff = (const int*)(beta + (size_t)ncols * k);
  cudaStream_t s = h->stream;
  k_lz_bounds<<<1, 256, 0, s>>>(ncols, k, alpha, beta, keff, h->d.scal);
  SQ_LAUNCH_CHECK(h);
  return set_bounds_device(h);   // no host round trip: the whole evaluation can be graph-captured
}

// set_bounds on the device, from the Lanczos interval scal[8], scal[9]: the step coefficients
// ca = 2 / zeta, cb = -2 chi / zeta, cd = ca lap0 + cb (SQ_MIXED: FP32-exact ca and cb, cd rounded
// once) and the effective interval the recurrence realises (centre moved by the stored
// stencil's constant-mode offset and cd's rounding) in scal[0], scal[1], scal[4..6]. Explicit
// rounding intrinsics keep every product and sum separately rounded, as in set_bounds.
__global__ void k_set_bounds(double* __restrict__ scal, double lap0, double lap_offset, int mixed, int* __restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double lo = scal[8], hi = scal[9];
  if (!(lo < hi) || !isfinite(lo) || !isfinite(hi)) {
    status[kStBadBounds] = 1;
    return;
  }
  status[kStBadBounds] = 0;
  double chi = __dmul_rn(0.5, __dadd_rn(hi, lo)), zeta = __dmul_rn(0.5, __dsub_rn(hi, lo));
  double ca = __ddiv_rn(2.0, zeta), cb = __ddiv_rn(__dmul_rn(-2.0, chi), zeta);
  if (mixed) {
    ca = double(__double2float_rn(ca));
    zeta = __ddiv_rn(2.0, ca);
    cb = double(__double2float_rn(__ddiv_rn(__dmul_rn(-2.0, chi), zeta)));
    chi = __ddiv_rn(__dmul_rn(-cb, zeta), 2.0);
  }
  const double exact = __dadd_rn(__dmul_rn(ca, lap0), cb);
  const double cd = mixed ? double(__double2float_rn(exact)) : exact;
  const double eps = __dsub_rn(cd, exact);
  chi = __dsub_rn(chi, __dadd_rn(lap_offset, __ddiv_rn(eps, ca)));
  scal[0] = __dsub_rn(chi, zeta);
  scal[1] = __dadd_rn(chi, zeta);
  scal[4] = ca;
  scal[5] = cb;
  scal[6] = cd;
}

int set_bounds_device(sq_handle* h) {
  k_set_bounds<<<1, 32, 0, h->stream>>>(h->d.scal, h->geo.lap0, h->lap_offset, h->precision == SQ_MIXED, h->d.status);
  SQ_LAUNCH_CHECK(h);
  return SQ_OK;
}

// Per-node bounds: every node column of the handle's tiles, in waves of nlz_wave tiles.
template <typename Real>
static int run_lanczos_nodes_t(sq_handle* h) {
  const Geo& g = h->geo;
  const int k = h->lanczos_k;
  for (int t0 = h->tile_begin; t0 < h->tile_end; t0 += h->nlz_wave) {
    const Wave w{t0, std::min(h->nlz_wave, h->tile_end - t0), nullptr};
    int rc = lanczos_columns<Real>(h, w, 0, k, reinterpret_cast<Real*>(h->d.nV), reinterpret_cast<Real*>(h->d.nW),
                                   reinterpret_cast<Real*>(h->d.nP), h->d.nC, &h->wb);
    if (rc != SQ_OK) return rc;
    const int ncols = w.ntiles * g.B;
    const double* alpha = h->d.nC + (size_t)3 * ncols * (k + 1);
    const double* beta = alpha + (size_t)ncols * k;
    const int* keff = (const int*)(beta + (size_t)ncols * k);
    k_lz_node_bounds<<<(ncols + 63) / 64, 64, 0, h->stream>>>(g, w, k, alpha, beta, keff, h->precision == SQ_MIXED,
                                                               h->lap_offset, h->d.nbnd, h->d.ncoef);
    SQ_LAUNCH_CHECK(h);
  }
  // the extreme node bounds (sq_get_bounds)
  std::vector<double> b(2 * size_t(h->Nd));
  SQ_CUDA_TRY(h, cudaMemcpyAsync(b.data(), h->d.nbnd, sizeof(double) * b.size(), cudaMemcpyDeviceToHost, h->stream));
  SQ_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  double lo = INFINITY, hi = -INFINITY;
  for (int q = 0; q < h->Nd; ++q) {
    if (!(b[2 * q] < b[2 * q + 1]) || !std::isfinite(b[2 * q]) || !std::isfinite(b[2 * q + 1]))
      return fail(h, SQ_ERR_CUDA, "per-node Lanczos bounds are not finite");
    lo = std::min(lo, b[2 * q]);
    hi = std::max(hi, b[2 * q + 1]);
  }
  h->lam_lo = lo;
  h->lam_hi = hi;
  return SQ_OK;
}

int run_lanczos_nodes(sq_handle* h) {
  if (h->lanczos_k + 1 > kMaxLanczosVecs) return fail(h, SQ_ERR_INVALID_ARG, "lanczos_k too large");
  if (h->precision == SQ_MIXED) return run_lanczos_nodes_t<float>(h);
  return run_lanczos_nodes_t<double>(h);
}

int run_lanczos(sq_handle* h) {
  if (h->lanczos_k + 1 > kMaxLanczosVecs) return fail(h, SQ_ERR_INVALID_ARG, "lanczos_k too large");
  if (h->precision == SQ_MIXED) return run_lanczos_t<float>(h);
  return run_lanczos_t<double>(h);
}

}  // namespace sq
