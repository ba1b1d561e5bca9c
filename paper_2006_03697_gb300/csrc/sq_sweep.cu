// The Chebyshev sweep of Sec. 4 over node tiles: for j = 0..n_pl
//     t^{j+1} = 2 Hhat_q t^j - t^{j-1}     (t^1 = Hhat_q t^0),   Hhat_q = (H_q - chi I) / zeta
// with H_q t = -1/2 sum_a (D2_a / h_a^2) t + V_eff t + sum_rows gamma |dOmega| chi (chi^T t),
// and the per-node moments rho^j, K^j_ab, N^j, S^j_ab of each column.
//
// Kernels (Real = double for SQ_FP64, float for SQ_MIXED; node sums always FP64):
//   k_stencil   one block per (z-slab of 4 planes, tile): H t^j on the union window, the
//               window mask, the recurrence update, and the fused nonlocal-stress partial
//               sum_u W_b (grad_a t^j) (the grad taps reuse the Laplacian's loads).
//   k_project   one block per (atom image, tile): P[row][q] = chi_row^T t^{j+1}.
//   k_moments   one warp per node: rho^j, K^j (restricted grad_a grad_b at the node),
//               N^j = sum_rows A P, S^j = sum of the slab partials; FP64 table row.
#include <algorithm>

#include "sq_device.cuh"

namespace sq {

template <typename Real>
struct Coef {
  Real ca, cb, cc;
};

template <typename Real>
__global__ void __launch_bounds__(kThreads)
k_stencil(Geo g, Wave w, const Real* __restrict__ Tc, const Real* __restrict__ Tp, Real* __restrict__ Tn,
          const Real* __restrict__ P, const Real* __restrict__ Wt, const Real* __restrict__ chi,
          const AtomTab* __restrict__ atoms, const double* __restrict__ chs, const TileEntry* __restrict__ entries,
          const int* __restrict__ blist, const int* __restrict__ bn, const Real* __restrict__ v,
          const double* __restrict__ scal, int mode, double* __restrict__ Spart) {
  // mode 0: t^1 = Hhat t^0;  mode 1: t^{j+1} = 2 Hhat t^j - t^{j-1};  mode 2: moments only;
  // mode 3: Tn = H_q t (restricted, unscaled; used by the Lanczos bounds)
  const int slab = blockIdx.x, tl = blockIdx.y, t = wave_tile(w, tl);
  int o[3];
  tile_origin(g, t, o);
  // step coefficients 2/zeta and -2 chi/zeta (halved for t^1 = Hhat t^0)
  const double f = (mode == 0) ? 0.5 : 1.0;
  const Real ca = Real(f * scal[4]), cb = Real(f * scal[5]), cc = Real(mode == 0 ? 0.0 : 1.0);
  const int Ux = g.U[0], Uy = g.U[1], Uz = g.U[2], B = g.B;
  const size_t tbase = (size_t)tl * g.Upts * B;
  const Real* T = Tc + tbase;
  const Real* Pt = P + (size_t)tl * g.r_cap * B;
  const TileEntry* ent = entries + (size_t)tl * g.e_cap;
  const int z0 = slab * kBrick, nz = min(kBrick, Uz - z0);
  const int nel = Ux * Uy * nz * B;
  const int sx = B, sy = Ux * B, sz = Ux * Uy * B;

  Real lap[3][kMaxNo + 1], grd[3][kMaxNo + 1];
  for (int a = 0; a < 3; ++a)
    for (int p = 0; p <= kMaxNo; ++p) {
      lap[a][p] = Real(g.lap[a][p]);
      grd[a][p] = Real(g.grd[a][p]);
    }
  const Real lap0 = Real(g.lap0);

  const int q = threadIdx.x % B;   // kThreads is a multiple of B: each thread keeps one node
  int qo[3];
  node_offset(g, q, qo);
  const bool valid = node_valid(g, o, qo);
  Real sacc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) sacc[k] = Real(0);

  for (int i = threadIdx.x; i < nel; i += kThreads) {
    const int p = i / B;
    const int ux = p % Ux, uy = (p / Ux) % Uy, uz = z0 + p / (Ux * Uy);
    const int pt = (uz * Uy + uy) * Ux + ux;
    const size_t e = (size_t)pt * B + q;
    if (!valid || !in_window(g, qo, ux, uy, uz)) {
      if (mode != 2) Tn[tbase + e] = Real(0);
      continue;
    }
    const Real tc = T[e];
    Real y = lap0 * tc;
    Real gr[3] = {Real(0), Real(0), Real(0)};
    const int u[3] = {ux, uy, uz};
    const int st[3] = {sx, sy, sz};
    const int Ua[3] = {Ux, Uy, Uz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      for (int pp = 1; pp <= g.n_o; ++pp) {
        const Real fp = (u[a] + pp < Ua[a]) ? T[e + (size_t)pp * st[a]] : Real(0);
        const Real fm = (u[a] - pp >= 0) ? T[e - (size_t)pp * st[a]] : Real(0);
        y += lap[a][pp] * (fp + fm);
        gr[a] += grd[a][pp] * (fp - fm);
      }
    }
    const int ax = o[0] - g.m[0] + ux, ay = o[1] - g.m[1] + uy, az = o[2] - g.m[2] + uz;
    {
      int wx = ax % g.n[0]; if (wx < 0) wx += g.n[0];
      int wy = ay % g.n[1]; if (wy < 0) wy += g.n[1];
      int wz = az % g.n[2]; if (wz < 0) wz += g.n[2];
      y += v[(wz * g.n[1] + wy) * g.n[0] + wx] * tc;
    }
    // nonlocal: sum over atom images covering this point of gamma |dOmega| chi(u) P[row][q]
    {
      const int br = ((uz / kBrick) * g.nbr[1] + uy / kBrick) * g.nbr[0] + ux / kBrick;
      const int* lst = blist + ((size_t)tl * g.nbricks + br) * g.br_cap;
      const int nb = bn[(size_t)tl * g.nbricks + br];
      for (int k = 0; k < nb; ++k) {
        const TileEntry te = ent[lst[k]];
        const AtomTab at = atoms[te.atom];
        const int li = box_index(at, te.s, g.n, ax, ay, az);
        if (li < 0) continue;
        const int boxpts = at.dim[0] * at.dim[1] * at.dim[2];
        for (int c = 0; c < at.nch; ++c)
          y += Real(chs[6 * (at.ch0 + c)]) * chi[at.off + (long long)c * boxpts + li] * Pt[(size_t)(te.row0 + c) * B + q];
      }
    }
    if (mode == 3) {          // plain H t (Lanczos)
      Tn[tbase + e] = y;
      continue;
    }
    if (mode != 2) {
      const Real tp = (mode == 1) ? Tp[tbase + e] : Real(0);
      Tn[tbase + e] = ca * y + cb * tc - cc * tp;
    }
    // S^j_ab partial: W_b(u, q) (grad_a t^j)(u)
    const Real* Wq = Wt + (size_t)tl * 3 * g.Upts * B;
    const Real w0 = Wq[e], w1 = Wq[(size_t)g.Upts * B + e], w2 = Wq[(size_t)2 * g.Upts * B + e];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      sacc[3 * a + 0] += gr[a] * w0;
      sacc[3 * a + 1] += gr[a] * w1;
      sacc[3 * a + 2] += gr[a] * w2;
    }
  }
  if (mode == 3) return;
  // deterministic block reduction per node: threads q, q + B, q + 2B, ... in order
  __shared__ double red[kThreads][9];
#pragma unroll
  for (int k = 0; k < 9; ++k) red[threadIdx.x][k] = double(sacc[k]);
  __syncthreads();
  for (int k2 = threadIdx.x; k2 < B * 9; k2 += kThreads) {
    const int qq = k2 / 9, k = k2 % 9;
    double s = 0.0;
    for (int th = qq; th < kThreads; th += B) s += red[th][k];
    Spart[(((size_t)tl * g.nslab + slab) * B + qq) * 9 + k] = s;
  }
}

template <typename Real>
__global__ void __launch_bounds__(kThreads)
k_project(Geo g, Wave w, const Real* __restrict__ Tn, const Real* __restrict__ chi, const AtomTab* __restrict__ atoms,
          const TileEntry* __restrict__ entries, const int* __restrict__ n_entries, Real* __restrict__ P) {
  const int eidx = blockIdx.x, tl = blockIdx.y, t = wave_tile(w, tl);
  if (eidx >= n_entries[tl]) return;
  int o[3];
  tile_origin(g, t, o);
  const TileEntry te = entries[(size_t)tl * g.e_cap + eidx];
  const AtomTab at = atoms[te.atom];
  const int B = g.B;
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    const int blo = at.lo[a] + te.s[a] * g.n[a] - (o[a] - g.m[a]);   // box corner in U-local coords
    lo[a] = max(0, blo);
    hi[a] = min(g.U[a], blo + at.dim[a]);
  }
  const int nx = max(0, hi[0] - lo[0]), ny = max(0, hi[1] - lo[1]), nzz = max(0, hi[2] - lo[2]);
  const int nel = nx * ny * nzz * B;
  const int boxpts = at.dim[0] * at.dim[1] * at.dim[2];
  const Real* T = Tn + (size_t)tl * g.Upts * B;
  const int q = threadIdx.x % B;
  Real acc[kMaxCh];
#pragma unroll
  for (int c = 0; c < kMaxCh; ++c) acc[c] = Real(0);
  for (int i = threadIdx.x; i < nel; i += kThreads) {
    const int p = i / B;
    const int lx = lo[0] + p % nx, ly = lo[1] + (p / nx) % ny, lz = lo[2] + p / (nx * ny);
    const Real tv = T[((size_t)(lz * g.U[1] + ly) * g.U[0] + lx) * B + q];
    if (tv == Real(0)) continue;
    const int li = box_index(at, te.s, g.n, o[0] - g.m[0] + lx, o[1] - g.m[1] + ly, o[2] - g.m[2] + lz);
#pragma unroll
    for (int c = 0; c < kMaxCh; ++c)
      if (c < at.nch) acc[c] += chi[at.off + (long long)c * boxpts + li] * tv;
  }
  __shared__ double red[kThreads][kMaxCh];
#pragma unroll
  for (int c = 0; c < kMaxCh; ++c) red[threadIdx.x][c] = double(acc[c]);
  __syncthreads();
  Real* Pt = P + (size_t)tl * g.r_cap * B;
  for (int k2 = threadIdx.x; k2 < B * at.nch; k2 += kThreads) {
    const int qq = k2 % B, c = k2 / B;
    double s = 0.0;
    for (int th = qq; th < kThreads; th += B) s += red[th][c];
    Pt[(size_t)(te.row0 + c) * B + qq] = Real(s);
  }
}

__constant__ int c_kpairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};

template <typename Real>
__global__ void __launch_bounds__(kThreads)
k_moments(Geo g, Wave w, int j, const Real* __restrict__ Tj, const Real* __restrict__ A, const Real* __restrict__ P,
          const int* __restrict__ n_rows, const double* __restrict__ Spart, double* __restrict__ mom) {
  const int tl = blockIdx.x, t = wave_tile(w, tl);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int o[3];
  tile_origin(g, t, o);
  const int B = g.B;
  const Real* T = Tj + (size_t)tl * g.Upts * B;
  const Real* At = A + (size_t)tl * g.r_cap * B;
  const Real* Pt = P + (size_t)tl * g.r_cap * B;
  const int nr = n_rows[tl];
  for (int q = warp; q < B; q += kThreads / 32) {
    int qo[3];
    node_offset(g, q, qo);
    if (!node_valid(g, o, qo)) continue;
    const int node = (o[0] + qo[0]) + g.n[0] * ((o[1] + qo[1]) + g.n[1] * (o[2] + qo[2]));
    const int c[3] = {qo[0] + g.m[0], qo[1] + g.m[1], qo[2] + g.m[2]};
    auto tval = [&](int x, int y, int z) -> double {
      if ((unsigned)x >= (unsigned)g.U[0] || (unsigned)y >= (unsigned)g.U[1] || (unsigned)z >= (unsigned)g.U[2]) return 0.0;
      return double(T[((size_t)(z * g.U[1] + y) * g.U[0] + x) * B + q]);
    };
    double out[SQ_N_MOMENTS];
    out[0] = tval(c[0], c[1], c[2]);
    // K^j_ab = [grad_a,q grad_b,q t^j]_q with both factors restricted to the window
    for (int pr = 0; pr < 6; ++pr) {
      const int a = c_kpairs[pr][0], b = c_kpairs[pr][1];
      double term = 0.0;
      if (lane < 2 * g.n_o) {
        const int pp = lane / 2 + 1;
        const int sg = (lane % 2 == 0) ? 1 : -1;
        if (pp <= g.m[a]) {
          int k[3] = {c[0], c[1], c[2]};
          k[a] += sg * pp;
          double gb = 0.0;
          for (int p2 = 1; p2 <= g.n_o; ++p2) {
            int kp[3] = {k[0], k[1], k[2]}, km[3] = {k[0], k[1], k[2]};
            kp[b] += p2;
            km[b] -= p2;
            gb += g.grd[b][p2] * (tval(kp[0], kp[1], kp[2]) - tval(km[0], km[1], km[2]));
          }
          term = sg * g.grd[a][pp] * gb;
        }
      }
      out[1 + pr] = warp_sum(term);
    }
    double nacc = 0.0;
    for (int r = lane; r < nr; r += 32) nacc += double(At[(size_t)r * B + q]) * double(Pt[(size_t)r * B + q]);
    out[7] = warp_sum(nacc);
    double sv = 0.0;
    if (lane < 9)
      for (int sl = 0; sl < g.nslab; ++sl) sv += Spart[(((size_t)tl * g.nslab + sl) * B + q) * 9 + lane];
    for (int k = 0; k < 9; ++k) out[8 + k] = __shfl_sync(0xffffffffu, sv, k);
    if (lane < SQ_N_MOMENTS) {
      double val = 0.0;
#pragma unroll
      for (int k = 0; k < SQ_N_MOMENTS; ++k)
        if (k == lane) val = out[k];
      mom[((size_t)node * (g.n_pl + 1) + j) * SQ_N_MOMENTS + lane] = val;
    }
  }
}

template <typename Real>
static int sweep_t(sq_handle* h, const Real* chi, const Real* v) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  Real* T[3] = {(Real*)h->wb.T[0], (Real*)h->wb.T[1], (Real*)h->wb.T[2]};
  Real* P = (Real*)h->wb.P;
  Real* A = (Real*)h->wb.A;
  Real* W = (Real*)h->wb.W;
  for (const Wave& w : h->waves) {
    int rc = build_wave_lists(h, w);
    if (rc != SQ_OK) return rc;
    const dim3 gstencil(g.nslab, w.ntiles), gproj(g.e_cap, w.ntiles);
    // algorithmic bytes of one stencil launch: node columns x region points x vectors moved
    long long nodes = 0;
    for (int tl = 0; tl < w.ntiles; ++tl) {
      const int t = w.tile0 + tl;
      const int o[3] = {(t % g.tiles[0]) * g.b, ((t / g.tiles[0]) % g.tiles[1]) * g.b,
                        (t / (g.tiles[0] * g.tiles[1])) * g.b};
      nodes += (long long)std::min(g.b, g.n[0] - o[0]) * std::min(g.b, g.n[1] - o[1]) * std::min(g.b, g.n[2] - o[2]);
    }
    const double col_bytes = double(nodes) * (2 * g.m[0] + 1) * (2 * g.m[1] + 1) * (2 * g.m[2] + 1) * sizeof(Real);
    cudaEvent_t ev = timing_begin(h, SQ_K_PROJECT, 0.0);
    k_project<Real><<<gproj, kThreads, 0, s>>>(g, w, T[0], chi, h->d.atoms, h->wb.entries, h->wb.n_entries, P);
    timing_end(h, ev);
    SQ_LAUNCH_CHECK(h);
    for (int j = 0; j <= g.n_pl; ++j) {
      Real* Tc = T[j % 3];
      Real* Tn = T[(j + 1) % 3];
      Real* Tp = T[(j + 2) % 3];
      const int mode = (j == g.n_pl) ? 2 : (j == 0 ? 0 : 1);
      const double vecs = (mode == 0) ? 2.0 : (mode == 1) ? 3.0 : 1.0;   // reads t^j (t^{j-1}), writes t^{j+1}
      ev = timing_begin(h, SQ_K_STENCIL, vecs * col_bytes);
      k_stencil<Real><<<gstencil, kThreads, 0, s>>>(g, w, Tc, Tp, Tn, P, W, chi, h->d.atoms, h->d.gdv, h->wb.entries,
                                                     h->wb.brick_list, h->wb.brick_n, v, h->d.scal, mode,
                                                     h->wb.Spart);
      timing_end(h, ev);
      SQ_LAUNCH_CHECK(h);
      ev = timing_begin(h, SQ_K_MOMENTS, 0.0);
      k_moments<Real><<<w.ntiles, kThreads, 0, s>>>(g, w, j, Tc, A, P, h->wb.n_rows, h->wb.Spart, h->d.mom);
      timing_end(h, ev);
      SQ_LAUNCH_CHECK(h);
      if (j < g.n_pl) {
        ev = timing_begin(h, SQ_K_PROJECT, 0.0);
        k_project<Real><<<gproj, kThreads, 0, s>>>(g, w, Tn, chi, h->d.atoms, h->wb.entries, h->wb.n_entries, P);
        timing_end(h, ev);
        SQ_LAUNCH_CHECK(h);
      }
    }
  }
  {
    int rc = timing_collect(h);
    if (rc != SQ_OK) return rc;
  }
  int st[kStCount];
  SQ_CUDA_TRY(h, cudaMemcpyAsync(st, h->d.status, sizeof(st), cudaMemcpyDeviceToHost, s));
  SQ_CUDA_TRY(h, cudaStreamSynchronize(s));
  if (st[kStOverflow]) return fail(h, SQ_ERR_CUDA, "internal list capacity exceeded");
  return SQ_OK;
}

int launch_apply_h64(sq_handle* h, const Wave& w, const double* v, double* out, double* P) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  k_project<double><<<dim3(g.e_cap, w.ntiles), kThreads, 0, s>>>(g, w, v, h->d.chi64, h->d.atoms, h->wb.entries,
                                                                  h->wb.n_entries, P);
  SQ_LAUNCH_CHECK(h);
  k_stencil<double><<<dim3(g.nslab, w.ntiles), kThreads, 0, s>>>(g, w, v, nullptr, out, P, nullptr, h->d.chi64,
                                                                  h->d.atoms, h->d.gdv, h->wb.entries, h->wb.brick_list,
                                                                  h->wb.brick_n, h->d.v64, h->d.scal, 3, nullptr);
  SQ_LAUNCH_CHECK(h);
  return SQ_OK;
}

int run_sweep(sq_handle* h) {
  if (h->precision == SQ_FP64) return sweep_t<double>(h, h->d.chi64, h->d.v64);
  return sweep_t<float>(h, h->d.chi32, h->d.v32);
}

}  // namespace sq
