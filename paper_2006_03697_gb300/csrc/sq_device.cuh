// Device-side helpers shared by the SQ kernels.
#pragma once

#include "sq_internal.h"

namespace sq {

__device__ __forceinline__ int floor_div_d(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int ceil_div_d(int a, int b) { return -floor_div_d(-a, b); }

// Tile t (global index) -> origin of its first node in lattice coordinates.
__device__ __forceinline__ void tile_origin(const Geo& g, int t, int o[3]) {
  o[0] = (t % g.tiles[0]) * g.b;
  o[1] = ((t / g.tiles[0]) % g.tiles[1]) * g.b;
  o[2] = (t / (g.tiles[0] * g.tiles[1])) * g.b;
}

__device__ __forceinline__ int wave_tile(const Wave& w, int tl) { return w.ids ? w.ids[tl] : w.tile0 + tl; }

// Node slot q of a tile -> offsets inside the tile.
__device__ __forceinline__ void node_offset(const Geo& g, int q, int qo[3]) {
  qo[0] = q % g.b;
  qo[1] = (q / g.b) % g.b;
  qo[2] = q / (g.b * g.b);
}

__device__ __forceinline__ bool node_valid(const Geo& g, const int o[3], const int qo[3]) {
  return o[0] + qo[0] < g.n[0] && o[1] + qo[1] < g.n[1] && o[2] + qo[2] < g.n[2];
}

// Is U-local point (ux, uy, uz) inside the window of the node with offsets qo?
__device__ __forceinline__ bool in_window(const Geo& g, const int qo[3], int ux, int uy, int uz) {
  return (unsigned)(ux - qo[0]) <= (unsigned)(2 * g.m[0]) &&
         (unsigned)(uy - qo[1]) <= (unsigned)(2 * g.m[1]) &&
         (unsigned)(uz - qo[2]) <= (unsigned)(2 * g.m[2]);
}

// x = hi + lo with hi, lo TF32 values (11 significant bits each, held in FP32 registers)
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
  const float r = x - __uint_as_float(hi);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

// d (16 x 8, FP32) += a (16 x 8, TF32, row) * b (8 x 8, TF32, col); fragment of lane (g, t),
// g = lane / 4, t = lane % 4: a = {(g, t), (g + 8, t), (g, t + 4), (g + 8, t + 4)},
// b = {(t, g), (t + 4, g)}, d = {(g, 2t), (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1)}
__device__ __forceinline__ void mma_tf32(float d[4], const uint32_t a[4], const uint32_t b[2]) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Linear index of an absolute lattice point inside an atom image's support box, or -1.
__device__ __forceinline__ int box_index(const AtomTab& at, const int s[3], const int n[3],
                                         int ax, int ay, int az) {
  int lx = ax - s[0] * n[0] - at.lo[0];
  int ly = ay - s[1] * n[1] - at.lo[1];
  int lz = az - s[2] * n[2] - at.lo[2];
  if ((unsigned)lx >= (unsigned)at.dim[0] || (unsigned)ly >= (unsigned)at.dim[1] ||
      (unsigned)lz >= (unsigned)at.dim[2])
    return -1;
  return (lz * at.dim[1] + ly) * at.dim[0] + lx;
}

// Pointer to the channel group of box point li of an atom's table.
template <typename Real>
__device__ __forceinline__ const Real* chi_row(const Real* chi, const AtomTab& at, int li) {
  return chi + at.off + (long long)li * at.nchp;
}

// Exclusive block-wide scan of one int per thread (blockDim.x a multiple of 32, <= 1024).
// Deterministic; returns the exclusive prefix and writes the block total to *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < nw) ? warp_sums[lane] : 0;
    for (int d = 1; d < 32; d <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    warp_sums[lane] = w;   // inclusive
  }
  __syncthreads();
  int excl = x - v + (warp > 0 ? warp_sums[warp - 1] : 0);
  *total = warp_sums[nw - 1];
  __syncthreads();
  return excl;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}


// Fermi-Dirac occupation 1 / (1 + e^x), evaluated without overflow for any x.
__device__ __forceinline__ double fermi_occ(double x) {
  const double ex = exp(-fabs(x));
  return (x > 0.0) ? ex / (1.0 + ex) : 1.0 / (1.0 + ex);
}

// Deterministic block sum (blockDim.x a power of two, sh holds blockDim.x doubles).
__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// N(mu) = 2 sum'_j c^j(mu) R^j = (4/M) sum_k g((chi + zeta cos theta_k - mu) / kT) F_k with
// F_k = sum'_j cos(j theta_k) R^j, theta_k = pi (k + 1/2) / M (the M-point Chebyshev-Gauss rule
// for the coefficient integral of Sec. 4). Whole block; same value in every thread.
__device__ __forceinline__ double electron_count_F(const double* F, int M, double chi_q, double zeta_q, double kT,
                                                  double mu, double* sh) {
  double s = 0.0;
  for (int k = threadIdx.x; k < M; k += blockDim.x)
    s += fermi_occ((chi_q + zeta_q * cos(M_PI * (k + 0.5) / M) - mu) / kT) * F[k];
  return 4.0 / M * block_sum_d(s, sh);
}

// The Fermi-level rule of the library: bisection on N(mu) = N_e over
// [lam_lo - 40 kT, lam_hi + 40 kT] until the bracket is < 1e-13 max(1, |mu|) or 200 steps, mu =
// the final midpoint. Returns false (and leaves *mu alone) when N(mu) - N_e has no sign change
// on the bracket. Whole block (sh: blockDim.x doubles); every thread gets the same result.
__device__ __forceinline__ bool fermi_bisect_rule(const double* F, int M, double lam_lo, double lam_hi, double kT,
                                                  double n_e, double* sh, double* mu) {
  const double chi_q = 0.5 * (lam_hi + lam_lo), zeta_q = 0.5 * (lam_hi - lam_lo);
  double lo = lam_lo - 40.0 * kT, hi = lam_hi + 40.0 * kT;
  const double nlo = electron_count_F(F, M, chi_q, zeta_q, kT, lo, sh);
  const double nhi = electron_count_F(F, M, chi_q, zeta_q, kT, hi, sh);
  if (!(nlo < n_e && n_e < nhi)) return false;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (electron_count_F(F, M, chi_q, zeta_q, kT, mid, sh) < n_e) lo = mid;
    else hi = mid;
    if (hi - lo < 1e-13 * fmax(1.0, fabs(mid))) break;
  }
  *mu = 0.5 * (lo + hi);
  return true;
}

}  // namespace sq
