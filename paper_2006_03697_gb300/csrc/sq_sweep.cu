// The Chebyshev sweep of Sec. 4 over node tiles: for j = 0..n_pl
//     t^{j+1} = 2 Hhat_q t^j - t^{j-1}     (t^1 = Hhat_q t^0),   Hhat_q = (H_q - chi I) / zeta
// with H_q t = -1/2 sum_a (D2_a / h_a^2) t + V_eff t + sum_rows gamma |dOmega| chi (chi^T t),
// and the per-node moments rho^j, K^j_ab, N^j, S^j_ab of each column.
//
// Kernels (Real = double for SQ_FP64, float for SQ_MIXED; node sums always FP64):
//   k_step      one block per (z-slab of 4 planes, tile), 4..8 warps; each warp walks whole
//               4^3 bricks, so the atom-image records of a brick (table offset, 64-bit mask of
//               the points inside the support sphere) are warp-uniform. Per brick:
//               A  the nonlocal apply sum_rows chi_row(u) Pg^j (Pg^j staged in shared memory);
//                  SQ_MIXED: a TF32 tensor-core product over the brick (3-term hi/lo split,
//                  tables stored pre-split), SQ_FP64: scalar and record-major;
//               B  Laplacian + V + the apply, the window mask, the recurrence update and the
//                  nonlocal-stress partial sum_u W_b (grad_a t^j) (the gradient taps reuse the
//                  Laplacian loads); SQ_MIXED: two nodes per lane (8-byte loads);
//               C  fused, the projections gamma |dOmega| chi^T t^{j+1} of the new column
//                  (SQ_MIXED: the transposed tensor-core product; SQ_FP64: register sums and a
//                  reduce-scatter over the point lanes), one shared-memory FP64 add per
//                  (image, channel, node), one global add per row and node per slab.
//   k_moments   one block per tile: rho^j, K^j (restricted grad_a grad_b at the node),
//               N^j = sum_rows chi(x_q) Pg^j, S^j = sum of the slab partials; FP64 table
//               row; then clears Pg^j, which accumulates the projections of step j + 1.
//   k_apply_h / k_project   plain H_q v for the Lanczos bounds (sweep precision).
#include <algorithm>

#include "sq_device.cuh"

namespace sq {

// ------------------------------------------------------------------------------ Lanczos apply
// P[row][q] = gamma |dOmega| chi_row^T v (one block per atom image of a tile)
template <typename Real>
__global__ void __launch_bounds__(kThreads)
k_project(Geo g, Wave w, const Real* __restrict__ Tn, const Real* __restrict__ chi, const AtomTab* __restrict__ atoms,
          const double* __restrict__ chs, const TileEntry* __restrict__ entries, const int* __restrict__ n_entries,
          Real* __restrict__ P) {
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
  const Real* T = Tn + (size_t)tl * g.Upts * B;
  Real acc[kMaxCh];
#pragma unroll
  for (int c = 0; c < kMaxCh; ++c) acc[c] = Real(0);
  for (int i = threadIdx.x; i < nel; i += kThreads) {
    const int p = i / B, q = i % B;
    const int lx = lo[0] + p % nx, ly = lo[1] + (p / nx) % ny, lz = lo[2] + p / (nx * ny);
    const Real tv = T[((size_t)(lz * g.U[1] + ly) * g.U[0] + lx) * B + q];
    if (tv == Real(0)) continue;
    const int li = box_index(at, te.s, g.n, o[0] - g.m[0] + lx, o[1] - g.m[1] + ly, o[2] - g.m[2] + lz);
    const Real* cr = chi_row(chi, at, li);
#pragma unroll
    for (int c = 0; c < kMaxCh; ++c)
      if (c < at.nch) acc[c] += cr[c] * tv;
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
    Pt[(size_t)(te.row0 + c) * B + qq] = Real(s * chs[6 * (at.ch0 + c)]);
  }
}

// out = H_q v on every node window of the wave (zero outside the windows); P from k_project. One
// block per (brick row: 4 y- and 4 z-planes of the window, all x; tile), so the few sample tiles
// of the Lanczos bounds still spread over the GPU.
template <typename Real>
__global__ void __launch_bounds__(kThreads)
k_apply_h(Geo g, Wave w, const Real* __restrict__ Tc, Real* __restrict__ Tn, const Real* __restrict__ P,
          const Real* __restrict__ chi, const AtomTab* __restrict__ atoms, const TileEntry* __restrict__ entries,
          const int* __restrict__ blist, const int* __restrict__ bn, const Real* __restrict__ v) {
  const int row = blockIdx.x, tl = blockIdx.y, t = wave_tile(w, tl);
  int o[3];
  tile_origin(g, t, o);
  const int Ux = g.U[0], Uy = g.U[1], Uz = g.U[2], B = g.B;
  const size_t tbase = (size_t)tl * g.Upts * B;
  const Real* T = Tc + tbase;
  const Real* Pt = P + (size_t)tl * g.r_cap * B;
  const TileEntry* ent = entries + (size_t)tl * g.e_cap;
  const int z0 = (row / g.nbr[1]) * kBrick, nz = min(kBrick, Uz - z0);
  const int y0 = (row % g.nbr[1]) * kBrick, ny = min(kBrick, Uy - y0);
  const int nel = Ux * ny * nz * B;
  const int st[3] = {B, Ux * B, Ux * Uy * B};
  const int Ua[3] = {Ux, Uy, Uz};
  for (int i = threadIdx.x; i < nel; i += kThreads) {
    const int p = i / B, q = i % B;
    int qo[3];
    node_offset(g, q, qo);
    const int ux = p % Ux, uy = y0 + (p / Ux) % ny, uz = z0 + p / (Ux * ny);
    const size_t e = (size_t)((uz * Uy + uy) * Ux + ux) * B + q;
    if (!node_valid(g, o, qo) || !in_window(g, qo, ux, uy, uz)) {
      Tn[tbase + e] = Real(0);
      continue;
    }
    const Real tc = T[e];
    Real y = Real(g.lap0) * tc;
    const int u[3] = {ux, uy, uz};
    for (int a = 0; a < 3; ++a)
      for (int pp = 1; pp <= g.n_o; ++pp) {
        const Real fp = (u[a] + pp < Ua[a]) ? T[e + (size_t)pp * st[a]] : Real(0);
        const Real fm = (u[a] - pp >= 0) ? T[e - (size_t)pp * st[a]] : Real(0);
        y += Real(g.lap[a][pp]) * (fp + fm);
      }
    const int ax = o[0] - g.m[0] + ux, ay = o[1] - g.m[1] + uy, az = o[2] - g.m[2] + uz;
    int wx = ax % g.n[0]; if (wx < 0) wx += g.n[0];
    int wy = ay % g.n[1]; if (wy < 0) wy += g.n[1];
    int wz = az % g.n[2]; if (wz < 0) wz += g.n[2];
    y += v[(wz * g.n[1] + wy) * g.n[0] + wx] * tc;
    const int br = ((uz / kBrick) * g.nbr[1] + uy / kBrick) * g.nbr[0] + ux / kBrick;
    const int* lst = blist + ((size_t)tl * g.nbricks + br) * g.br_cap;
    const int nb = bn[(size_t)tl * g.nbricks + br];
    for (int k = 0; k < nb; ++k) {
      const TileEntry te = ent[lst[k]];
      const AtomTab at = atoms[te.atom];
      const int li = box_index(at, te.s, g.n, ax, ay, az);
      if (li < 0) continue;
      const Real* cr = chi_row(chi, at, li);
      for (int c = 0; c < at.nch; ++c) y += cr[c] * Pt[(size_t)(te.row0 + c) * B + q];
    }
    Tn[tbase + e] = y;
  }
}

// ------------------------------------------------------------------------------ sweep step
// stencil weights of the sweep's precision, read straight from the kernel parameters
template <typename Real> struct Coef;
template <> struct Coef<float> {
  static __device__ __forceinline__ float lap0(const Geo& g) { return g.lap0f; }
  static __device__ __forceinline__ float lap(const Geo& g, int a, int p) { return g.lapf[a][p]; }
  static __device__ __forceinline__ float grd(const Geo& g, int a, int p) { return g.grdf[a][p]; }
};
template <> struct Coef<double> {
  static __device__ __forceinline__ double lap0(const Geo& g) { return g.lap0; }
  static __device__ __forceinline__ double lap(const Geo& g, int a, int p) { return g.lap[a][p]; }
  static __device__ __forceinline__ double grd(const Geo& g, int a, int p) { return g.grd[a][p]; }
};

template <typename Real> struct V4;
template <> struct V4<float> { using T = float4; };
template <> struct V4<double> { using T = double4_32a; };

template <typename Real>
__device__ __forceinline__ void load4(const Real* p, Real out[4]) {
  const typename V4<Real>::T x = *reinterpret_cast<const typename V4<Real>::T*>(p);
  out[0] = x.x;
  out[1] = x.y;
  out[2] = x.z;
  out[3] = x.w;
}

constexpr int kTileB = 8;   // nodes per tile (2 x 2 x 2); one warp = 4 points x 8 nodes

// ---- warp-level TF32 tensor-core products for the FP32 projector phases.
// x = hi + lo with hi, lo TF32 (11 significant bits each); a product is taken as
// hi*hi + hi*lo + lo*hi with FP32 accumulation (the lo*lo term, ~2^-22 relative, is dropped).

// (mma_tf32: the warp-level m16n8k8 TF32 product, sq_device.cuh)

__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// the brick's t values in the per-warp shared array: point p = a + 4 b + 16 c, node q
__device__ __forceinline__ int tn_index(int p, int q) { return (p >> 2) * 32 + (p & 3) * kTileB + q; }

// mode 0: t^1 = Hhat t^0;  mode 1: t^{j+1} = 2 Hhat t^j - t^{j-1};  mode 2: moments only.
// Each warp walks whole 4^3 bricks of the slab: iteration it covers brick points
// (a, b, c) = (lane >> 3, it & 3, it >> 2) for node q = lane & 7, so the 4 x-points of an
// iteration are contiguous in memory and every image record is warp-uniform.
// kSmemP: stage Pg^j and accumulate the slab's projections in shared memory (false when a
// tile has too many projector rows; Pg^j is then read and Pg^{j+1} accumulated in global memory)
constexpr int kStepThreads = 256;   // most threads of a k_step block (its warps walk the slab's bricks)

// Warps per k_step block: 4..8, the count that leaves the fewest idle warp-turns over the
// slab's bricks (49 bricks -> 7 warps, 16 -> 8, 36 -> 6); ties go to more warps.
static int step_warps(int bricks_per_slab) {
  int best = kStepThreads / 32, idle_best = 1 << 30;
  for (int w = kStepThreads / 32; w >= 4; --w) {
    const int idle = (bricks_per_slab + w - 1) / w * w - bricks_per_slab;
    if (idle < idle_best) {
      idle_best = idle;
      best = w;
    }
  }
  return best;
}

template <typename Real, int NO, bool kSmemP, bool kMMA>
__global__ void __launch_bounds__(kStepThreads, sizeof(Real) == 4 ? 4 : 2)
k_step(Geo g, Wave w, const Real* __restrict__ Tc, const Real* __restrict__ Tp, Real* __restrict__ Tn,
       const double* __restrict__ Pg, double* __restrict__ Pg_next, const Real* __restrict__ Wt,
       const Real* __restrict__ chi, const float* __restrict__ chis, const Real* __restrict__ gdv,
       const int4* __restrict__ brec, const int* __restrict__ slab_n, const int* __restrict__ slab_map, const int* __restrict__ bn,
       const Real* __restrict__ v, const double* __restrict__ scal, int mode, double* __restrict__ Spart,
       int rows_smem, const double* __restrict__ ncoef, int* __restrict__ status) {
  // dynamic shared memory: [Ps: rows_smem x 8 FP64][red: nw x 8 x 9 FP64][Pstage: rows_smem x 8]
  // [tn_sm: nw x 16 x 32] (Ps and Pstage only with kSmemP; rows_smem = 0 otherwise)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // wrapped V_eff index contributions of the slab's x, y and z positions (cell is periodic)
  __shared__ int wrx[kMaxU], wry[kBrick], wrz[kMaxU];
  const int slab = blockIdx.x, tl = blockIdx.y, t = wave_tile(w, tl);
  double* Pn = Pg_next + (size_t)tl * g.r_cap * kTileB;
  // projections of t^{j+1}, summed in FP64 ([slab rows][8]); Pg^j staged in the sweep precision.
  // In shared memory only the rows of the images that meet this slab are held (slab-local
  // numbering, smap: slab row -> tile row); without it records index the tile rows directly.
  double* Ps = kSmemP ? reinterpret_cast<double*>(smem_raw) : Pn;
  const int nsr = kSmemP ? slab_n[(size_t)tl * g.nslab + slab] : 0;
  if (kSmemP && nsr > rows_smem) {   // a launch sized for another layout (e.g. a stale graph): refuse
    if (threadIdx.x == 0) atomicOr(status + kStOverflow, 4);
    return;
  }
  const int* smap = slab_map + ((size_t)tl * g.nslab + slab) * g.r_cap;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* red = reinterpret_cast<double*>(smem_raw) + (size_t)rows_smem * kTileB;        // S partials [nw][8][9]
  Real* Pstage = reinterpret_cast<Real*>(red + nw * kTileB * 9);
  Real* tn_sm = Pstage + (size_t)rows_smem * kTileB;                                      // [nw][16][32]
  int o[3];
  tile_origin(g, t, o);
  const double f = (mode == 0) ? 0.5 : 1.0;
  // step coefficients: off-diagonal ca = 2/zeta, diagonal cd = ca lap0 + cb (cb = -2 chi/zeta)
  const Real ca = Real(f * scal[4]), cd = Real(f * scal[6]), cc = Real(mode == 0 ? 0.0 : 1.0);
  const int Ux = g.U[0], Uy = g.U[1], Uz = g.U[2];
  const size_t tbase = (size_t)tl * g.Upts * kTileB;
  const Real* T = Tc + tbase;
  const double* Pt = Pg + (size_t)tl * g.r_cap * kTileB;
  const bool project = (mode != 2);
  const int st[3] = {kTileB, Ux * kTileB, Ux * Uy * kTileB};
  const int Ua[3] = {Ux, Uy, Uz};
  for (int i = threadIdx.x; i < g.U[0] + kBrick + g.U[2]; i += blockDim.x) {
    int a, u;
    if (i < g.U[0]) { a = 0; u = i; }
    else if (i < g.U[0] + kBrick) { a = 1; u = slab * kBrick + i - g.U[0]; }
    else { a = 2; u = i - g.U[0] - kBrick; }
    int wv = (o[a] - g.m[a] + u) % g.n[a];
    if (wv < 0) wv += g.n[a];
    if (a == 0) wrx[u] = wv;
    else if (a == 1) wry[u - slab * kBrick] = wv * g.n[0];
    else wrz[u] = wv * g.n[0] * g.n[1];
  }
  if (kSmemP) {
    for (int i = threadIdx.x; i < nsr * kTileB; i += blockDim.x) {
      Pstage[i] = Real(Pt[smap[i >> 3] * kTileB + (i & 7)]);
      if (project) Ps[i] = 0.0;
    }
  }
  __syncthreads();
  // without shared memory the apply reads Pg^j from global memory (FP64) directly
  auto pg = [&](int idx) -> Real { return kSmemP ? Pstage[idx] : Real(Pt[idx]); };

  const int q = lane & 7, pa = lane >> 3;
  int qo[3];
  qo[0] = q & 1;
  qo[1] = (q >> 1) & 1;
  qo[2] = q >> 2;
  const bool valid = node_valid(g, o, qo);
  // step coefficients of the lane's node(s): the block's (shared bounds) or each node's own
  // (per-node bounds; paired phase: nodes 2 np2 and 2 np2 + 1, scalar phase: node q)
  Real caA = ca, cdA = cd, caB = ca, cdB = cd;
  if (ncoef) {
    auto own = [&](int qx, int qy, int qz, Real& c_a, Real& c_d) {
      const int qq[3] = {qx, qy, qz};
      if (!node_valid(g, o, qq)) return;
      const int node = (o[0] + qx) + g.n[0] * ((o[1] + qy) + g.n[1] * (o[2] + qz));
      c_a = Real(f * ncoef[2 * node]);
      c_d = Real(f * ncoef[2 * node + 1]);
    };
    if constexpr (kMMA) {
      const int p2 = lane & 3;
      own(0, p2 & 1, p2 >> 1, caA, cdA);
      own(1, p2 & 1, p2 >> 1, caB, cdB);
    } else {
      own(qo[0], qo[1], qo[2], caA, cdA);
    }
  }
  const Real* Wq = Wt + (size_t)tl * 3 * g.Upts * kTileB;
  const size_t wstr = (size_t)g.Upts * kTileB;
  // S partial sums: per lane across bricks (scalar path); the paired phase B reduces them per
  // brick over its point lanes into a per-warp FP32 array (red, read as floats), so no S
  // registers stay live through the projector phases
  Real sacc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) sacc[k] = Real(0);
  float* red32 = reinterpret_cast<float*>(red) + warp * kTileB * 9;
  if constexpr (kMMA) {
    for (int k = lane; k < kTileB * 9; k += 32) red32[k] = 0.f;
    __syncwarp();
  }
  // paired phase B: lane = node pair np2 (nodes 2 np2, 2 np2 + 1: x offsets 0 and 1), x-point xa2,
  // y parity yb2
  const int np2 = lane & 3, xa2 = (lane >> 2) & 3, yb2 = lane >> 4;
  const int qo2[3] = {0, np2 & 1, np2 >> 1};
  bool valid2[2];
  {
    int qa[3] = {0, qo2[1], qo2[2]}, qb[3] = {1, qo2[1], qo2[2]};
    valid2[0] = node_valid(g, o, qa);
    valid2[1] = node_valid(g, o, qb);
  }
  const int nbx = g.nbr[0], nby = g.nbr[1], nbz = g.nbr[2];

  for (int bi = warp; bi < nbx * nbz; bi += nw) {
    const int bx = bi % nbx, bz = bi / nbx, by = slab;
    const int br = (bz * nby + by) * nbx + bx;
    const int4* rb = brec + ((size_t)tl * g.nbricks + br) * g.br_cap * 2;
    const int nb = bn[(size_t)tl * g.nbricks + br];
    Real* tnv = tn_sm + warp * 16 * 32 + lane;   // per lane and brick point: V_nl t^j, then t^{j+1}
    if constexpr (kMMA) {
      // phase A on tensor cores: Y[64 points][8 nodes] = X[64 points][4 nb rows] Pg^j[4 nb rows][8],
      // X = the brick's projector values (zero outside each image's sphere). M = brick points
      // (m-tile = one z-plane), N = the 8 nodes, K = 2 images x 4 channels per k-step, ordered so
      // that each lane's A and B elements are two adjacent channels of one image:
      // K = t -> (image k2 + t / 2, channel 2 (t % 2)), K = t + 4 -> the next channel.
      const int g8 = lane >> 2, t4 = lane & 3, ch = 2 * (t4 & 1);
      const int pa0 = g8 & 3, pb0 = g8 >> 2;         // lane's rows: points (pa0, pb0, c), (pa0, pb0 + 2, c)
      float acc[4][4];
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[mt][i] = 0.f;
      for (int k2 = 0; k2 < nb; k2 += 2) {
        const int kr = k2 + (t4 >> 1);
        int4 r0 = make_int4(0, 0, 0, 0), r1 = make_int4(0, 0, 0, 0);
        if (kr < nb) {
          r0 = rb[2 * kr];
          r1 = rb[2 * kr + 1];
        }
        const int nch = r0.w & 0xff, prow = int(unsigned(r0.w) >> 16);
        const float p0 = (ch < nch) ? float(Pstage[(prow + ch) * kTileB + g8]) : 0.f;
        const float p1 = (ch + 1 < nch) ? float(Pstage[(prow + ch + 1) * kTileB + g8]) : 0.f;
        uint32_t bh[2], bl[2];
        split_tf32(p0, bh[0], bl[0]);
        split_tf32(p1, bh[1], bl[1]);
        const int dx = r1.x, plane = r1.x * r1.y * 4;
        // (hi, lo) pairs of channels ch, ch + 1 at point (pa0, pb0, 0): one 16-byte load per point
        // (FP32 values split in the kernel instead halve these bytes but measured 3.5 % slower)
        const float* xb = chis + 2 * (r0.x + (pb0 * dx + pa0) * 4 + ch);
        const unsigned mlo = unsigned(r1.z) >> g8, mhi = unsigned(r1.w) >> g8;
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
          const unsigned mw = (mt < 2) ? mlo : mhi;
          const int sh = 16 * (mt & 1);
          uint4 x0 = make_uint4(0u, 0u, 0u, 0u), x1 = make_uint4(0u, 0u, 0u, 0u);
          if ((mw >> sh) & 1u) x0 = *reinterpret_cast<const uint4*>(xb + 2 * mt * plane);
          if ((mw >> (sh + 8)) & 1u) x1 = *reinterpret_cast<const uint4*>(xb + 2 * (mt * plane + 8 * dx));
          const uint32_t ah[4] = {x0.x, x1.x, x0.z, x1.z}, al[4] = {x0.y, x1.y, x0.w, x1.w};
          mma_tf32(acc[mt], al, bh);   // small terms first
          mma_tf32(acc[mt], ah, bl);
          mma_tf32(acc[mt], ah, bh);
        }
      }
      Real* tw = tn_sm + warp * 16 * 32;
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int i = 0; i < 4; ++i) tw[tn_index(16 * mt + g8 + 8 * (i >> 1), 2 * t4 + (i & 1))] = Real(acc[mt][i]);
    } else {
      // phase A: nonlocal apply, record-major: sum_rows chi_row(u) Pg^j[row][q] for the lane's
      // 16 points; the table loads of one record are independent of each other
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {        // 8 points at a time keeps the accumulators in registers
        Real ynl[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) ynl[i] = Real(0);
        for (int k = 0; k < nb; ++k) {
          const int4 r0 = rb[2 * k], r1 = rb[2 * k + 1];
          const int nch = r0.w & 0xff, nchp = (r0.w >> 8) & 0xff;
          const int prow = kSmemP ? (int(unsigned(r0.w) >> 16)) : r0.y;
          const unsigned mk = unsigned(half ? r1.w : r1.z) >> pa;   // bits pa + 4 i of this half
          if (!(mk & 0x11111111u)) continue;
          for (int c0 = 0; c0 < nch; c0 += 4) {
            Real pv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) pv[c] = (c0 + c < nch) ? pg((prow + c0 + c) * kTileB + q) : Real(0);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              if ((mk >> (4 * i)) & 1u) {
                const int it = 8 * half + i;
                Real cv[4];
                load4(chi + r0.x + (((it >> 2) * r1.y + (it & 3)) * r1.x + pa) * nchp + c0, cv);
                ynl[i] += cv[0] * pv[0] + cv[1] * pv[1] + cv[2] * pv[2] + cv[3] * pv[3];
              }
            }
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) tnv[(8 * half + i) * 32] = ynl[i];
      }
    }
    __syncwarp();
    if constexpr (kMMA) {
      // phase B with two nodes per lane: lane = (node pair np, x-point xa, y parity yb); iteration
      // it covers brick points (xa, 2 (it % 2) + yb, it / 2) for nodes 2 np and 2 np + 1, so every
      // t / W load is an 8-byte pair and a brick takes 8 iterations (half the load round trips)
      Real* tw = tn_sm + warp * 16 * 32;
      float sb[18];   // S partials of nodes 2 np2 and 2 np2 + 1 over this brick
#pragma unroll
      for (int k = 0; k < 18; ++k) sb[k] = 0.f;
#pragma unroll 1
      for (int it = 0; it < 8; ++it) {
        const int pb = 2 * (it & 1) + yb2, pc = it >> 1;
        const int ux = bx * kBrick + xa2, uy = by * kBrick + pb, uz = bz * kBrick + pc;
        const int p = xa2 + 4 * pb + 16 * pc;
        const bool inU = (uy < Uy) && (uz < Uz);
        const size_t e = (size_t)((uz * Uy + uy) * Ux + ux) * kTileB + 2 * np2;
        const bool inyz = inU && (unsigned)(uy - qo2[1]) <= (unsigned)(2 * g.m[1]) &&
                          (unsigned)(uz - qo2[2]) <= (unsigned)(2 * g.m[2]);
        const bool in0 = inyz && valid2[0] && (unsigned)ux <= (unsigned)(2 * g.m[0]);
        const bool in1 = inyz && valid2[1] && (unsigned)(ux - 1) <= (unsigned)(2 * g.m[0]);
        float2 tn = make_float2(0.f, 0.f);
        if (in0 || in1) {
          const float2 w0 = ld2(Wq + e), w1 = ld2(Wq + wstr + e), w2 = ld2(Wq + 2 * wstr + e);
          const float2 tp = (mode == 1) ? ld2(Tp + tbase + e) : make_float2(0.f, 0.f);
          const float2 tc = ld2(T + e);
          float2 y = make_float2(0.f, 0.f);           // off-diagonal part of H t^j
          float2 gr[3];
          const int u[3] = {ux, uy, uz};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            gr[a] = make_float2(0.f, 0.f);
#pragma unroll
            for (int pp = 1; pp <= NO; ++pp) {
              const float2 fp = (u[a] + pp < Ua[a]) ? ld2(T + e + (size_t)pp * st[a]) : make_float2(0.f, 0.f);
              const float2 fm = (u[a] - pp >= 0) ? ld2(T + e - (size_t)pp * st[a]) : make_float2(0.f, 0.f);
              const float wl = Coef<float>::lap(g, a, pp), wg = Coef<float>::grd(g, a, pp);
              y.x += wl * (fp.x + fm.x);
              y.y += wl * (fp.y + fm.y);
              gr[a].x += wg * (fp.x - fm.x);
              gr[a].y += wg * (fp.y - fm.y);
            }
          }
          const float vloc = float(v[wrz[uz] + wry[pb] + wrx[ux]]);
          const float2 ynl = *reinterpret_cast<const float2*>(tw + tn_index(p, 2 * np2));   // phase A
          y.x += ynl.x;
          y.y += ynl.y;
          if (mode != 2) {
            const float dgA = float(cdA) + float(caA) * vloc, dgB = float(cdB) + float(caB) * vloc;
            if (in0) tn.x = float(caA) * y.x + dgA * tc.x - float(cc) * tp.x;
            if (in1) tn.y = float(caB) * y.y + dgB * tc.y - float(cc) * tp.y;
            *reinterpret_cast<float2*>(Tn + tbase + e) = tn;
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) {   // W is zero outside each node's window
            sb[3 * a + 0] += gr[a].x * w0.x;
            sb[3 * a + 1] += gr[a].x * w1.x;
            sb[3 * a + 2] += gr[a].x * w2.x;
            sb[9 + 3 * a + 0] += gr[a].y * w0.y;
            sb[9 + 3 * a + 1] += gr[a].y * w1.y;
            sb[9 + 3 * a + 2] += gr[a].y * w2.y;
          }
        } else if (inU && mode != 2) {
          *reinterpret_cast<float2*>(Tn + tbase + e) = tn;
        }
        *reinterpret_cast<float2*>(tw + tn_index(p, 2 * np2)) = tn;
      }
      // the brick's S partials: sum over the 8 point lanes of each node pair, lanes 0..3 add
#pragma unroll
      for (int k = 0; k < 18; ++k) {
        float sv = sb[k];
        sv += __shfl_xor_sync(0xffffffffu, sv, 4);
        sv += __shfl_xor_sync(0xffffffffu, sv, 8);
        sv += __shfl_xor_sync(0xffffffffu, sv, 16);
        if (lane < 4) red32[(2 * lane + k / 9) * 9 + k % 9] += sv;
      }
    } else {
#pragma unroll 1
      for (int it = 0; it < 16; ++it) {
        const int pb = it & 3, pc = it >> 2;
        const int ux = bx * kBrick + pa, uy = by * kBrick + pb, uz = bz * kBrick + pc;
        const bool inU = (uy < Uy) && (uz < Uz);
        const size_t e = (size_t)((uz * Uy + uy) * Ux + ux) * kTileB + q;
        const bool inwin = inU && valid && in_window(g, qo, ux, uy, uz);
        Real tn = Real(0);
        if (inwin) {
          // loads that do not depend on the stencil, issued first
          const Real w0 = Wq[e], w1 = Wq[wstr + e], w2 = Wq[2 * wstr + e];
          const Real tp = (mode == 1) ? Tp[tbase + e] : Real(0);
          const Real tc = T[e];
          Real y = Real(0);                           // off-diagonal part of H t^j
          Real gr[3];
          const int u[3] = {ux, uy, uz};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            gr[a] = Real(0);
#pragma unroll
            for (int pp = 1; pp <= NO; ++pp) {
              const Real fp = (u[a] + pp < Ua[a]) ? T[e + (size_t)pp * st[a]] : Real(0);
              const Real fm = (u[a] - pp >= 0) ? T[e - (size_t)pp * st[a]] : Real(0);
              y += Coef<Real>::lap(g, a, pp) * (fp + fm);
              gr[a] += Coef<Real>::grd(g, a, pp) * (fp - fm);
            }
          }
          const Real vloc = v[wrz[uz] + wry[pb] + wrx[ux]];   // V_eff at the wrapped node
          y += tnv[it * 32];                          // nonlocal part from phase A
          if (mode != 2) {
            tn = caA * y + (cdA + caA * vloc) * tc - cc * tp;
            Tn[tbase + e] = tn;
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            sacc[3 * a + 0] += gr[a] * w0;
            sacc[3 * a + 1] += gr[a] * w1;
            sacc[3 * a + 2] += gr[a] * w2;
          }
        } else if (inU && mode != 2) {
          Tn[tbase + e] = Real(0);
        }
        tnv[it * 32] = tn;
      }
    }
    __syncwarp();
    // projections of t^{j+1} over this brick: each lane sums its 16 points in registers, a
    // reduce-scatter over the 4 x-point lanes (xor 8, then xor 16) leaves lane (pa, q) with the
    // brick sum of channel c0 + pa for node q, so one FP64 conversion and one shared add per
    // lane cover 4 channels x 8 nodes (FP64 instructions are narrow on this part)
    if constexpr (kMMA) {
      if (project) {
        // phase C on tensor cores: Pg^{j+1}[4 nb rows][8] += X^T[4 nb rows][64 points] t^{j+1}[64][8].
        // M = 4 images x 4 channels per m-tile, ordered so each lane's A elements are two adjacent
        // channels of one image (row g -> image m4 + g / 2, channel 2 (g % 2); row g + 8 -> the
        // next channel), K = 8 brick points per k-step, N = the 8 nodes.
        const int g8 = lane >> 2, t4 = lane & 3, ch = 2 * (g8 & 1);
        const Real* tw = tn_sm + warp * 16 * 32;
        // one m-tile (4 images) per pass; separate accumulators for the three split terms
        // measured slower (more registers live across the gather loads), so one chain
        for (int m4 = 0; m4 < nb; m4 += 4) {
          const int kr = m4 + (g8 >> 1);
          int4 r0 = make_int4(0, 0, 0, 0), r1 = make_int4(0, 0, 0, 0);
          if (kr < nb) {
            r0 = rb[2 * kr];
            r1 = rb[2 * kr + 1];
          }
          const int dx = r1.x, dy = r1.y;
          const float* xb = chis + 2 * (r0.x + t4 * 4 + ch);   // (hi, lo) pairs at point (t4, 0, 0)
          const unsigned mlo = unsigned(r1.z) >> t4, mhi = unsigned(r1.w) >> t4;
          float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int ks = 0; ks < 8; ++ks) {
            // points p0 = 8 ks + t4 = (t4, 2 (ks % 2), ks / 2) and p1 = p0 + 4 (one row further in b)
            const unsigned mw = (ks < 4) ? mlo : mhi;
            const int sh = 8 * (ks & 3);
            const float* xp = xb + 2 * ((ks >> 1) * dy + 2 * (ks & 1)) * dx * 4;
            uint4 x0 = make_uint4(0u, 0u, 0u, 0u), x1 = make_uint4(0u, 0u, 0u, 0u);
            if ((mw >> sh) & 1u) x0 = *reinterpret_cast<const uint4*>(xp);
            if ((mw >> (sh + 4)) & 1u) x1 = *reinterpret_cast<const uint4*>(xp + 2 * dx * 4);
            const uint32_t ah[4] = {x0.x, x0.z, x1.x, x1.z}, al[4] = {x0.y, x0.w, x1.y, x1.w};
            uint32_t bh[2], bl[2];
            split_tf32(float(tw[tn_index(8 * ks + t4, g8)]), bh[0], bl[0]);
            split_tf32(float(tw[tn_index(8 * ks + t4 + 4, g8)]), bh[1], bl[1]);
            mma_tf32(d, al, bh);
            mma_tf32(d, ah, bl);
            mma_tf32(d, ah, bh);
          }
          const int nch = r0.w & 0xff, prow = int(unsigned(r0.w) >> 16);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int cc = ch + (i >> 1);
            if (cc < nch && d[i] != 0.f)
              atomicAdd(&Ps[(prow + cc) * kTileB + 2 * t4 + (i & 1)], double(d[i] * float(gdv[r0.z + cc])));
          }
        }
      }
    } else {
      if (project) {
        const bool b0 = (pa & 1) != 0, b1 = (pa & 2) != 0;
        for (int k = 0; k < nb; ++k) {
          const int4 r0 = rb[2 * k], r1 = rb[2 * k + 1];
          const int nch = r0.w & 0xff, nchp = (r0.w >> 8) & 0xff;
          const int prow = kSmemP ? (int(unsigned(r0.w) >> 16)) : r0.y;
          const unsigned mlo = unsigned(r1.z) >> pa, mhi = unsigned(r1.w) >> pa;
          for (int c0 = 0; c0 < nch; c0 += 4) {
            Real acc[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll 4
            for (int it = 0; it < 16; ++it) {
              const unsigned bit = ((it < 8 ? mlo : mhi) >> (4 * (it & 7))) & 1u;
              if (bit) {
                const Real tv = tnv[it * 32];
                Real cv[4];
                load4(chi + r0.x + (((it >> 2) * r1.y + (it & 3)) * r1.x + pa) * nchp + c0, cv);
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[c] += cv[c] * tv;
              }
            }
            // step 1 (pa bit 0): keep channels {b0, 2 + b0}, hand the other two to the partner
            Real k0 = b0 ? acc[1] : acc[0], k1 = b0 ? acc[3] : acc[2];
            const Real g0 = b0 ? acc[0] : acc[1], g1 = b0 ? acc[2] : acc[3];
            k0 += __shfl_xor_sync(0xffffffffu, g0, 8);
            k1 += __shfl_xor_sync(0xffffffffu, g1, 8);
            // step 2 (pa bit 1): keep channel b0 + 2 b1 = pa
            Real s = b1 ? k1 : k0;
            s += __shfl_xor_sync(0xffffffffu, b1 ? k0 : k1, 16);
            const int c = c0 + pa;
            if (c < nch && s != Real(0)) atomicAdd(&Ps[(prow + c) * kTileB + q], double(s * gdv[r0.z + c]));
          }
        }
      }
    }
  }
  // S partials: fixed-order reduction per node (the point lanes by shuffles, then warps)
  if constexpr (!kMMA) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double sv = double(sacc[k]);
      sv += __shfl_xor_sync(0xffffffffu, sv, 8);
      sv += __shfl_xor_sync(0xffffffffu, sv, 16);
      if (lane < kTileB) red[(warp * kTileB + lane) * 9 + k] = sv;
    }
  }
  __syncthreads();
  for (int k2 = threadIdx.x; k2 < kTileB * 9; k2 += blockDim.x) {
    const int qq = k2 / 9, k = k2 % 9;
    double sv = 0.0;
    for (int wv = 0; wv < nw; ++wv)
      sv += kMMA ? double(reinterpret_cast<const float*>(red)[(wv * kTileB + qq) * 9 + k])
                 : red[(wv * kTileB + qq) * 9 + k];
    Spart[(((size_t)tl * g.nslab + slab) * kTileB + qq) * 9 + k] = sv;
  }
  if (kSmemP && project) {
    for (int i = threadIdx.x; i < nsr * kTileB; i += blockDim.x) {
      const double s = Ps[i];
      if (s != 0.0) atomicAdd(&Pn[smap[i >> 3] * kTileB + (i & 7)], s);
    }
  }
}

__constant__ int c_kpairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};

// Moments of t^j per node (one warp per node), then Pg^j := 0 (the accumulator of step j + 1).
template <typename Real>
__global__ void __launch_bounds__(kThreads)
k_moments(Geo g, Wave w, int j, const Real* __restrict__ Tj, const Real* __restrict__ A, double* __restrict__ Pg,
          const int* __restrict__ n_rows, const double* __restrict__ Spart, double* __restrict__ mom) {
  const int tl = blockIdx.x, t = wave_tile(w, tl);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int o[3];
  tile_origin(g, t, o);
  const int B = g.B;
  const Real* T = Tj + (size_t)tl * g.Upts * B;
  const Real* At = A + (size_t)tl * g.r_cap * B;
  double* Pt = Pg + (size_t)tl * g.r_cap * B;
  const int nr = n_rows[tl];
  for (int q = warp; q < B; q += kThreads / 32) {
    int qo[3];
    node_offset(g, q, qo);
    if (!node_valid(g, o, qo)) continue;
    const int node = (o[0] + qo[0]) + g.n[0] * ((o[1] + qo[1]) + g.n[1] * (o[2] + qo[2]));
    const int c[3] = {qo[0] + g.m[0], qo[1] + g.m[1], qo[2] + g.m[2]};
    // FP64 arithmetic on the stored values: the restricted grad_a grad_a at the node cancels
    // strongly, and an FP32 version measured 4x the sigma^I error on the 216-atom instance
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
    // N^j = w_q^T V_nl,q t^j = sum_rows chi_row(x_q) (gamma |dOmega| chi_row^T t^j)
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
  __syncthreads();
  for (int i = threadIdx.x; i < nr * B; i += kThreads) Pt[i] = 0.0;
}

// dynamic shared memory of k_step: staged projections (at most kStepRowsSmemMax, else they stay
// in global memory) + the per-warp arrays
constexpr int kStepRowsSmemMax = 160 * 1024;
constexpr int kStepSmemMax = kStepRowsSmemMax + (kStepThreads / 32) * (kTileB * 9 * 8 + 16 * 32 * 8);

// largest projector-row count a step block stages in shared memory (more rows: global memory)
int step_rows_smem_max(int precision) {
  return int(kStepRowsSmemMax / (kTileB * (sizeof(double) + (precision == SQ_FP64 ? sizeof(double) : sizeof(float)))));
}

template <typename Real, int NO>
static int launch_step(sq_handle* h, const Wave& w, dim3 grid, size_t smem, const Real* Tc, const Real* Tp, Real* Tn,
                       const double* Pg, double* Pgn, const Real* W, const Real* chi, const Real* gdv, const Real* v,
                       int mode) {
  const int rows_smem = int(smem / (kTileB * (sizeof(double) + sizeof(Real))));
  const double* ncoef = (h->bounds_mode == SQ_BOUNDS_PER_NODE) ? h->d.ncoef : nullptr;
  const int nw = h->step_warps > 0 ? h->step_warps : step_warps(h->geo.nbr[0] * h->geo.nbr[2]), nthr = 32 * nw;
  const size_t smem_warps = size_t(nw) * (kTileB * 9 * sizeof(double) + 16 * 32 * sizeof(Real));
  // The dynamic-size attribute belongs to the function, not the launch, and handles on other
  // host threads launch the same kernel, so every caller sets the same value (the largest
  // dynamic size this kernel uses)
  if (rows_smem <= h->step_rows_cap) {
    smem += smem_warps;
    if (sizeof(Real) == 4 && h->proj4) {
      h->step_variant[0]++;
      SQ_CUDA_TRY(h, cudaFuncSetAttribute(k_step<Real, NO, true, sizeof(Real) == 4>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, kStepSmemMax));
      k_step<Real, NO, true, sizeof(Real) == 4><<<grid, nthr, smem, h->stream>>>(
          h->geo, w, Tc, Tp, Tn, Pg, Pgn, W, chi, h->d.chi32s, gdv, h->wb.brick_rec, h->wb.slab_n, h->wb.slab_map,
          h->wb.brick_n, v, h->d.scal, mode, h->wb.Spart, rows_smem, ncoef, h->d.status);
      SQ_LAUNCH_CHECK(h);
      return SQ_OK;
    }
    h->step_variant[1]++;
    SQ_CUDA_TRY(h, cudaFuncSetAttribute(k_step<Real, NO, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kStepSmemMax));
    k_step<Real, NO, true, false><<<grid, nthr, smem, h->stream>>>(h->geo, w, Tc, Tp, Tn, Pg, Pgn, W, chi, nullptr, gdv,
                                                                h->wb.brick_rec, h->wb.slab_n, h->wb.slab_map, h->wb.brick_n, v,
                                                                h->d.scal, mode, h->wb.Spart, rows_smem, ncoef, h->d.status);
  } else {
    h->step_variant[2]++;
    SQ_CUDA_TRY(h, cudaFuncSetAttribute(k_step<Real, NO, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kStepSmemMax));
    k_step<Real, NO, false, false><<<grid, nthr, smem_warps, h->stream>>>(h->geo, w, Tc, Tp, Tn, Pg, Pgn, W, chi, nullptr, gdv,
                                                              h->wb.brick_rec, h->wb.slab_n, h->wb.slab_map, h->wb.brick_n, v,
                                                              h->d.scal, mode, h->wb.Spart, 0, ncoef, h->d.status);
  }
  SQ_LAUNCH_CHECK(h);
  return SQ_OK;
}

template <typename Real>
static int dispatch_step(sq_handle* h, const Wave& w, dim3 grid, size_t smem, const Real* Tc, const Real* Tp, Real* Tn,
                         const double* Pg, double* Pgn, const Real* W, const Real* chi, const Real* gdv, const Real* v,
                         int mode) {
  switch (h->geo.n_o) {
    case 1: return launch_step<Real, 1>(h, w, grid, smem, Tc, Tp, Tn, Pg, Pgn, W, chi, gdv, v, mode);
    case 2: return launch_step<Real, 2>(h, w, grid, smem, Tc, Tp, Tn, Pg, Pgn, W, chi, gdv, v, mode);
    case 3: return launch_step<Real, 3>(h, w, grid, smem, Tc, Tp, Tn, Pg, Pgn, W, chi, gdv, v, mode);
    case 4: return launch_step<Real, 4>(h, w, grid, smem, Tc, Tp, Tn, Pg, Pgn, W, chi, gdv, v, mode);
    case 5: return launch_step<Real, 5>(h, w, grid, smem, Tc, Tp, Tn, Pg, Pgn, W, chi, gdv, v, mode);
    default: return launch_step<Real, 6>(h, w, grid, smem, Tc, Tp, Tn, Pg, Pgn, W, chi, gdv, v, mode);
  }
}

// images one stage of the TMA-staged step holds in wave wi: the wave's fullest brick, at most
// kStepTmaRecs (a brick with more takes them in chunks)
static int stage_recs(const sq_handle* h, size_t wi) {
  return std::max(1, std::min(h->wave_recs[wi], h->stage_recs_cap));
}

// The TMA-staged step (sq_step_tma.cu), when selected (SQ_STEP_KERNEL=staged), runs a mixed sweep
// wave when its maps exist and the slab's projections and one stage fit in shared memory.
static bool use_tma(const sq_handle* h, size_t wi) {
  if (!h->tma_ok || !h->step_staged || h->precision != SQ_MIXED) return false;
  if (wi >= h->wave_rows.size() || wi >= h->wave_recs.size()) return false;
  const int rows = std::max(1, h->wave_rows[wi]);
  if (rows > h->step_rows_cap) return false;   // the global-memory projection path
  return step_tma_smem_bytes(rows, stage_recs(h, wi)) <= kStepTmaSmemMax;
}

template <typename Real>
static int sweep_t(sq_handle* h, const Real* chi, const Real* v, const Real* gdv) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  Real* T[3] = {(Real*)h->wb.T[0], (Real*)h->wb.T[1], (Real*)h->wb.T[2]};
  double* Pg[2] = {(double*)h->wb.Pg[0], (double*)h->wb.Pg[1]};
  Real* A = (Real*)h->wb.A;
  Real* W = (Real*)h->wb.W;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SQ_CUDA_TRY(h, cudaStreamIsCapturing(s, &cap));
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  if (h->wave_rows.size() != h->waves.size() || h->wave_recs.size() != h->waves.size()) {
    if (capturing) return fail(h, SQ_ERR_STATE, "wave layout not measured before capture");
    int rc = measure_wave_rows(h);
    if (rc != SQ_OK) return rc;
  }
  for (size_t wi = 0; wi < h->waves.size(); ++wi) {
    NvtxRange nvtx("sweep wave");
    const Wave& w = h->waves[wi];
    // a captured graph must rebuild the lists itself (the atoms may move before it runs again)
    int rc = build_wave_lists(h, w, !capturing);
    if (rc != SQ_OK) return rc;
    // largest slab projector-row count of the wave (measured once per layout) sizes the
    // per-slab shared accumulator
    const int rmax = h->wave_rows[wi];
    const size_t smem = std::max<size_t>(1, size_t(rmax)) * kTileB * (sizeof(double) + sizeof(Real));

    const dim3 gstencil(g.nslab, w.ntiles);
    // algorithmic bytes of one stencil launch: node columns x region points x vectors moved
    long long nodes = 0;
    for (int tl = 0; tl < w.ntiles; ++tl) {
      const int t = w.tile0 + tl;
      const int o[3] = {(t % g.tiles[0]) * g.b, ((t / g.tiles[0]) % g.tiles[1]) * g.b,
                        (t / (g.tiles[0] * g.tiles[1])) * g.b};
      nodes += (long long)std::min(g.b, g.n[0] - o[0]) * std::min(g.b, g.n[1] - o[1]) * std::min(g.b, g.n[2] - o[2]);
    }
    const double col_bytes = double(nodes) * (2 * g.m[0] + 1) * (2 * g.m[1] + 1) * (2 * g.m[2] + 1) * sizeof(Real);
    for (int j = 0; j <= g.n_pl; ++j) {
      Real* Tc = T[j % 3];
      Real* Tn = T[(j + 1) % 3];
      Real* Tp = T[(j + 2) % 3];
      const int mode = (j == g.n_pl) ? 2 : (j == 0 ? 0 : 1);
      const double vecs = (mode == 0) ? 2.0 : (mode == 1) ? 3.0 : 1.0;   // reads t^j (t^{j-1}), writes t^{j+1}
      cudaEvent_t ev = capturing ? nullptr : timing_begin(h, SQ_K_STENCIL, vecs * col_bytes);
      if (sizeof(Real) == 4 && use_tma(h, wi))
        rc = launch_step_tma(h, w, gstencil, j % 3, (j + 2) % 3, (float*)Tn, Pg[j % 2], Pg[(j + 1) % 2], mode,
                             std::max(1, rmax), stage_recs(h, wi));
      else
        rc = dispatch_step<Real>(h, w, gstencil, smem, Tc, Tp, Tn, Pg[j % 2], Pg[(j + 1) % 2], W, chi, gdv, v, mode);
      if (rc != SQ_OK) return rc;
      timing_end(h, ev);
      ev = capturing ? nullptr : timing_begin(h, SQ_K_MOMENTS, 0.0);
      k_moments<Real><<<w.ntiles, kThreads, 0, s>>>(g, w, j, Tc, A, Pg[j % 2], h->wb.n_rows, h->wb.Spart, h->d.mom);
      timing_end(h, ev);
      SQ_LAUNCH_CHECK(h);
    }
  }
  if (capturing) return SQ_OK;   // the status words are read after the graph runs
  {
    int rc = timing_collect(h);
    if (rc != SQ_OK) return rc;
  }
  int st[kStCount];
  SQ_CUDA_TRY(h, cudaMemcpyAsync(st, h->d.status, sizeof(st), cudaMemcpyDeviceToHost, s));
  SQ_CUDA_TRY(h, cudaStreamSynchronize(s));
  if (st[kStOverflow]) return fail(h, SQ_ERR_CUDA, "internal list capacity exceeded");
  if (st[kStBadBounds]) return fail(h, SQ_ERR_CUDA, "spectral bounds are not finite or empty");
  if (st[kStTimeout]) return fail(h, SQ_ERR_TIMEOUT, "a staged step block's copy wait ran out");
  return SQ_OK;
}

template <typename Real>
static int time_step_t(sq_handle* h, int reps, double* ms_out, const Real* chi, const Real* v, const Real* gdv) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  if (h->waves.empty()) {
    *ms_out = 0.0;
    return SQ_OK;
  }
  if (h->wave_rows.size() != h->waves.size() || h->wave_recs.size() != h->waves.size()) {
    int rc = measure_wave_rows(h);
    if (rc != SQ_OK) return rc;
  }
  const Wave& w = h->waves[0];
  cudaEvent_t e0, e1;
  SQ_CUDA_TRY(h, cudaEventCreate(&e0));
  SQ_CUDA_TRY(h, cudaEventCreate(&e1));
  // a sweep rebuilds each wave's lists and W table (unless sq_keep_lists holds them for one wave):
  // that cost, spread over the sweep's n_pl + 1 steps, belongs to the step time the tuner compares
  const bool rebuilt = h->waves.size() > 1 || !h->keep_lists;
  cudaEventRecord(e0, s);
  int rc = build_wave_lists(h, w, !rebuilt);
  cudaEventRecord(e1, s);
  float ms_lists = 0.f;
  if (rc == SQ_OK && rebuilt && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms_lists, e0, e1);
  if (rc != SQ_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
  }
  Real* T[3] = {(Real*)h->wb.T[0], (Real*)h->wb.T[1], (Real*)h->wb.T[2]};
  double* Pg[2] = {(double*)h->wb.Pg[0], (double*)h->wb.Pg[1]};
  const size_t smem = std::max<size_t>(1, size_t(h->wave_rows[0])) * kTileB * (sizeof(double) + sizeof(Real));
  const dim3 grid(g.nslab, w.ntiles);
  const bool tma = sizeof(Real) == 4 && use_tma(h, 0);
  const int rows = std::max(1, h->wave_rows[0]), recs = stage_recs(h, 0);
  // the first launch (mode 0) forms t^1 from t^0, so the timed launches read defined values
  if (tma)
    rc = launch_step_tma(h, w, grid, 0, 2, (float*)T[1], Pg[0], Pg[1], 0, rows, recs);
  else
    rc = dispatch_step<Real>(h, w, grid, smem, T[0], T[2], T[1], Pg[0], Pg[1], (Real*)h->wb.W, chi, gdv, v, 0);
  if (rc != SQ_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
  }
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps && rc == SQ_OK; ++r)
    rc = tma ? launch_step_tma(h, w, grid, 1, 0, (float*)T[2], Pg[1], Pg[0], 1, rows, recs)
             : dispatch_step<Real>(h, w, grid, smem, T[1], T[0], T[2], Pg[1], Pg[0], (Real*)h->wb.W, chi, gdv, v, 1);
  cudaEventRecord(e1, s);
  float ms = 0.f;
  const cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SQ_OK) return rc;
  if (e != cudaSuccess) return fail(h, SQ_ERR_CUDA, std::string("step timing: ") + cudaGetErrorString(e));
  *ms_out = double(ms) / std::max(1, reps) + double(ms_lists) / (g.n_pl + 1);
  return SQ_OK;
}

int time_step_launch(sq_handle* h, int reps, double* ms_out) {
  if (h->precision == SQ_FP64) return time_step_t<double>(h, reps, ms_out, h->d.chi64, h->d.v64, h->d.gdv64);
  return time_step_t<float>(h, reps, ms_out, h->d.chi32, h->d.v32, h->d.gdv32);
}

int measure_wave_rows(sq_handle* h) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  std::vector<int> nrows, nrecs;
  h->wave_rows.assign(h->waves.size(), 0);
  h->wave_recs.assign(h->waves.size(), 0);
  for (size_t wi = 0; wi < h->waves.size(); ++wi) {
    const Wave& w = h->waves[wi];
    int rc = build_wave_entries(h, w);
    if (rc != SQ_OK) return rc;
    nrows.resize(size_t(w.ntiles) * g.nslab);
    nrecs.resize(size_t(w.ntiles) * g.nbricks);
    SQ_CUDA_TRY(h, cudaMemcpyAsync(nrows.data(), h->wb.slab_n, sizeof(int) * nrows.size(), cudaMemcpyDeviceToHost, s));
    SQ_CUDA_TRY(h, cudaMemcpyAsync(nrecs.data(), h->wb.brick_n, sizeof(int) * nrecs.size(), cudaMemcpyDeviceToHost, s));
    SQ_CUDA_TRY(h, cudaStreamSynchronize(s));
    h->wave_rows[wi] = nrows.empty() ? 0 : *std::max_element(nrows.begin(), nrows.end());
    h->wave_recs[wi] = nrecs.empty() ? 0 : *std::max_element(nrecs.begin(), nrecs.end());
  }
  return SQ_OK;
}

template <typename Real>
static int apply_h_t(sq_handle* h, const Wave& w, const Real* v, Real* out, Real* P, const Real* chi, const Real* vpot,
                     const WaveBufs& b) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  k_project<Real><<<dim3(g.e_cap, w.ntiles), kThreads, 0, s>>>(g, w, v, chi, h->d.atoms, h->d.gdv, b.entries,
                                                               b.n_entries, P);
  SQ_LAUNCH_CHECK(h);
  k_apply_h<Real><<<dim3(g.nbr[2] * g.nbr[1], w.ntiles), kThreads, 0, s>>>(g, w, v, out, P, chi, h->d.atoms, b.entries,
                                                               b.brick_list, b.brick_n, vpot);
  SQ_LAUNCH_CHECK(h);
  return SQ_OK;
}

int launch_apply_h(sq_handle* h, const Wave& w, const double* v, double* out, double* P, const WaveBufs& b) {
  return apply_h_t<double>(h, w, v, out, P, h->d.chi64, h->d.v64, b);
}

int launch_apply_h(sq_handle* h, const Wave& w, const float* v, float* out, float* P, const WaveBufs& b) {
  return apply_h_t<float>(h, w, v, out, P, h->d.chi32, h->d.v32, b);
}

int run_sweep(sq_handle* h) {
  if (h->precision == SQ_FP64) return sweep_t<double>(h, h->d.chi64, h->d.v64, h->d.gdv64);
  return sweep_t<float>(h, h->d.chi32, h->d.v32, h->d.gdv32);
}

}  // namespace sq
