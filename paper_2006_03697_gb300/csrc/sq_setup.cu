// Setup kernels: projector tables, per-tile atom-image lists, per-brick lists, the
// projector weights at the nodes (A) and the per-node nonlocal-stress weights (W).
//
// Projectors (Sec. 2, E_nl and sigma^III; Gaussian stand-ins):
//   chi_00 = (pi w^2)^(-3/4) exp(-r^2 / 2w^2),  chi_1m = sqrt(2)/w d_m (pi w^2)^(-3/4) exp(-r^2 / 2w^2)
// sampled at the absolute lattice points x = u h of each atom's support box (base image).
// A periodic image of the atom shifted by s cells uses the same table at u - s n.
#include "sq_device.cuh"

namespace sq {

// chs layout per channel: [gamma*dV, l, m, width, rcut, 0]
template <typename Real>
__global__ void k_chi_tables(Geo g, const AtomTab* __restrict__ atoms, const double* __restrict__ chs,
                             Real* __restrict__ chi) {
  const AtomTab at = atoms[blockIdx.x];
  const int boxpts = at.dim[0] * at.dim[1] * at.dim[2];
  for (int i = threadIdx.x; i < boxpts; i += blockDim.x) {
    const int lx = i % at.dim[0], ly = (i / at.dim[0]) % at.dim[1], lz = i / (at.dim[0] * at.dim[1]);
    const double d[3] = {(at.lo[0] + lx) * g.h[0] - at.R[0], (at.lo[1] + ly) * g.h[1] - at.R[1],
                         (at.lo[2] + lz) * g.h[2] - at.R[2]};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    for (int c = 0; c < at.nch; ++c) {
      const double* sp = chs + 6 * (at.ch0 + c);
      const int l = int(sp[1]), mch = int(sp[2]);
      const double w = sp[3], rc = sp[4];
      double val = 0.0;
      if (r2 <= rc * rc) {
        const double base = pow(M_PI * w * w, -0.75) * exp(-r2 / (2.0 * w * w));
        val = (l == 0) ? base : sqrt(2.0) / w * d[mch] * base;
      }
      chi[at.off + (long long)i * at.nchp + c] = Real(val);
    }
    for (int c = at.nch; c < at.nchp; ++c) chi[at.off + (long long)i * at.nchp + c] = Real(0);   // padding
  }
}

// out[2 i], out[2 i + 1] = TF32 (hi, lo) of in[i]: the tensor-core projector phases load a
// point's channel pair as one 16-byte (hi, lo, hi, lo) group
__global__ void k_split_tf32(const float* __restrict__ in, long long n, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    uint32_t hi, lo;
    split_tf32(in[i], hi, lo);
    out[2 * i] = __uint_as_float(hi);
    out[2 * i + 1] = __uint_as_float(lo);
  }
}

// One block per tile of the wave: list the atom images (atom, shift s) whose support box
// meets the tile's union window, atom-major then s (x fastest); assign projector rows.
__global__ void k_tile_entries(Geo g, Wave w, const AtomTab* __restrict__ atoms, TileEntry* __restrict__ entries,
                               int* __restrict__ n_entries, int* __restrict__ n_rows, int* __restrict__ status) {
  const int tl = blockIdx.x, t = wave_tile(w, tl);
  int o[3];
  tile_origin(g, t, o);
  int ulo[3], uhi[3];
  for (int a = 0; a < 3; ++a) {
    ulo[a] = o[a] - g.m[a];
    uhi[a] = ulo[a] + g.U[a] - 1;
  }
  TileEntry* out = entries + (size_t)tl * g.e_cap;
  int base_e = 0, base_r = 0;
  for (int a0 = 0; a0 < g.n_atoms; a0 += blockDim.x) {
    const int J = a0 + threadIdx.x;
    int cnt = 0, nch = 0, slo[3] = {0, 0, 0}, ns[3] = {0, 0, 0};
    if (J < g.n_atoms) {
      const AtomTab at = atoms[J];
      nch = at.nch;
      if (nch > 0 && at.dim[0] > 0 && at.dim[1] > 0 && at.dim[2] > 0) {
        cnt = 1;
        for (int a = 0; a < 3; ++a) {
          slo[a] = ceil_div_d(ulo[a] - (at.lo[a] + at.dim[a] - 1), g.n[a]);
          const int shi = floor_div_d(uhi[a] - at.lo[a], g.n[a]);
          ns[a] = max(0, shi - slo[a] + 1);
          cnt *= ns[a];
        }
      }
    }
    int tot_e, tot_r;
    const int off_e = block_exclusive_scan(cnt, &tot_e);
    const int off_r = block_exclusive_scan(cnt * nch, &tot_r);
    for (int k = 0; k < cnt; ++k) {
      const int idx = base_e + off_e + k;
      if (idx < g.e_cap && base_r + off_r + (k + 1) * nch <= g.r_cap) {
        TileEntry e;
        e.atom = J;
        e.s[0] = slo[0] + k % ns[0];
        e.s[1] = slo[1] + (k / ns[0]) % ns[1];
        e.s[2] = slo[2] + k / (ns[0] * ns[1]);
        e.row0 = base_r + off_r + k * nch;
        e.pad = 0;
        out[idx] = e;
      }
    }
    base_e += tot_e;
    base_r += tot_r;
  }
  if (threadIdx.x == 0) {
    const bool over = base_e > g.e_cap || base_r > g.r_cap;
    // on overflow nothing downstream may index past the capacities: empty lists, error flag
    n_entries[tl] = over ? 0 : base_e;
    n_rows[tl] = over ? 0 : base_r;
    if (over) atomicOr(status + kStOverflow, 1);
  }
}

// Support sphere of an atom image against a lattice box [bl, bhi] (absolute coords): the
// table box overlaps it and the distance from the image centre to its bounding box is <= rcut.
// FP32 on small, box-relative coordinates (FP64 instructions issue at a small fraction of FP32
// on this part) with a relative margin of 1e-5 on rcut^2, so the test never drops an image the
// FP64 table holds non-zero values for (an extra image only adds zeros).
__device__ __forceinline__ bool image_meets_box(const Geo& g, const TileEntry& te, const AtomTab& at, float rc,
                                                const int bl[3], const int bhi[3]) {
  bool hit = true;
  float d2 = 0.f;
  for (int a = 0; a < 3; ++a) {
    const int lo = at.lo[a] + te.s[a] * g.n[a], hi = lo + at.dim[a] - 1;
    hit = hit && (lo <= bhi[a]) && (hi >= bl[a]);
    // relative to the lattice point lo: image centre at -dlo, box from (bl - lo) h to (bhi - lo) h
    const float h = float(g.h[a]), c = -at.dlo[a];
    const float blo = float(bl[a] - lo) * h, bhx = float(bhi[a] - lo) * h;
    const float dd = (c < blo) ? blo - c : (c > bhx ? c - bhx : 0.f);
    d2 += dd * dd;
  }
  return hit && (d2 <= rc * rc * (1.f + 1e-5f) + 1e-10f);
}

// One warp per (brick, tile): entries whose support sphere meets the brick, in entry order,
// and their records. The projector rows of the entries that meet the brick's slab (its y-row
// of bricks: all of U in x and z, the brick's y-planes; a superset of its bricks' entries: the
// slab's bounding box contains each brick's) are numbered slab-locally in entry order; the
// record carries that number (bits 16..31 of r0.w) and the first brick of the slab writes the
// slab's row map (slab row -> tile row) and count.
__global__ void k_brick_lists(Geo g, Wave w, const AtomTab* __restrict__ atoms, const double* __restrict__ rcmax,
                              const TileEntry* __restrict__ entries, const int* __restrict__ n_entries,
                              int* __restrict__ blist, int* __restrict__ bn, int4* __restrict__ rec,
                              float4* __restrict__ d0, int4* __restrict__ tma, int* __restrict__ slab_n,
                              int* __restrict__ slab_map, int* __restrict__ status) {
  const int br = blockIdx.x, tl = blockIdx.y, t = wave_tile(w, tl), lane = threadIdx.x;
  int o[3];
  tile_origin(g, t, o);
  const int bx = br % g.nbr[0], by = (br / g.nbr[0]) % g.nbr[1], bz = br / (g.nbr[0] * g.nbr[1]);
  const int bl[3] = {o[0] - g.m[0] + bx * kBrick, o[1] - g.m[1] + by * kBrick, o[2] - g.m[2] + bz * kBrick};
  const int bhi[3] = {o[0] - g.m[0] + min(g.U[0], (bx + 1) * kBrick) - 1,
                      o[1] - g.m[1] + min(g.U[1], (by + 1) * kBrick) - 1,
                      o[2] - g.m[2] + min(g.U[2], (bz + 1) * kBrick) - 1};
  // the slab: all of U in x and z, the brick's planes in y
  const int sl[3] = {o[0] - g.m[0], bl[1], o[2] - g.m[2]};
  const int shi[3] = {o[0] - g.m[0] + g.U[0] - 1, bhi[1], o[2] - g.m[2] + g.U[2] - 1};
  const bool slab_writer = (bx == 0 && bz == 0);
  int* smap = slab_map + ((size_t)tl * g.nslab + by) * g.r_cap;
  const int ne = n_entries[tl];
  const TileEntry* ent = entries + (size_t)tl * g.e_cap;
  int* out = blist + ((size_t)tl * g.nbricks + br) * g.br_cap;
  int cnt = 0, srow_base = 0;
  for (int e0 = 0; e0 < ne; e0 += 32) {
    const int e = e0 + lane;
    bool hit = false;
    int nch_slab = 0;
    TileEntry te;
    AtomTab at;
    if (e < ne) {
      te = ent[e];
      at = atoms[te.atom];
      const float rcf = float(rcmax[te.atom]);
      hit = image_meets_box(g, te, at, rcf, bl, bhi);
      if (image_meets_box(g, te, at, rcf, sl, shi)) nch_slab = at.nch;
    }
    // slab-local first row of the lane's entry: exclusive warp scan of the slab entries' rows
    int incl = nch_slab;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    const int srow = srow_base + incl - nch_slab;
    if (slab_writer)
      for (int c = 0; c < nch_slab; ++c) smap[srow + c] = te.row0 + c;
    srow_base += __shfl_sync(0xffffffffu, incl, 31);
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    const int pos = cnt + __popc(mask & ((1u << lane) - 1u));
    if (hit && pos < g.br_cap) out[pos] = e;
    // one record per hit image, built by the whole warp: lane L tests brick points L and L + 32
    // (bit a + 4 b + 16 c) for lying in the brick, the box and the support sphere, with the same
    // arithmetic as the table (a point outside has all channels zero)
    for (unsigned hm = mask; hm; hm &= hm - 1u) {
      const int src = __ffs(hm) - 1;
      const int pos_s = cnt + __popc(mask & ((1u << src) - 1u));
      const int e_s = e0 + src;
      if (pos_s >= g.br_cap) break;
      const TileEntry tes = ent[e_s];
      const AtomTab ats = atoms[tes.atom];
      const int srow_s = __shfl_sync(0xffffffffu, srow, src);
      int l0[3];
      for (int a = 0; a < 3; ++a) l0[a] = bl[a] - (ats.lo[a] + tes.s[a] * g.n[a]);
      const float rc = float(rcmax[tes.atom]);
      bool inpt[2];
      for (int hh = 0; hh < 2; ++hh) {
        const int pbit = lane + 32 * hh;
        const int pl[3] = {pbit & 3, (pbit >> 2) & 3, pbit >> 4};
        bool in = true;
        float r2 = 0.f;
        for (int a = 0; a < 3; ++a) {
          const int l = l0[a] + pl[a];
          in = in && (bl[a] + pl[a] <= bhi[a]) && l >= 0 && l < ats.dim[a];
          const float d = float(l) * float(g.h[a]) + ats.dlo[a];   // (lo + l) h - R, box-relative
          r2 += d * d;
        }
        // superset of the table's non-zero points (FP32 with a 1e-5 margin on rcut^2)
        inpt[hh] = in && r2 <= rc * rc * (1.f + 1e-5f) + 1e-10f;
      }
      const unsigned lo32 = __ballot_sync(0xffffffffu, inpt[0]);
      const unsigned hi32 = __ballot_sync(0xffffffffu, inpt[1]);
      if (lane == 0) {
        const int offc = int(ats.off + (long long)((l0[2] * ats.dim[1] + l0[1]) * ats.dim[0] + l0[0]) * ats.nchp);
        int4* r = rec + (((size_t)tl * g.nbricks + br) * g.br_cap + pos_s) * 2;
        r[0] = make_int4(offc, tes.row0, ats.ch0, ats.nch | (ats.nchp << 8) | (min(srow_s, 0xffff) << 16));
        r[1] = make_int4(ats.dim[0], ats.dim[1], int(lo32), int(hi32));
        // x - R of the brick corner for this image, (lo + l0) h - R, formed in FP64 and rounded once
        // (once per record: the per-point work adds only the in-brick offset)
        d0[((size_t)tl * g.nbricks + br) * g.br_cap + pos_s] =
            make_float4(float((ats.lo[0] + l0[0]) * g.h[0] - ats.R[0]), float((ats.lo[1] + l0[1]) * g.h[1] - ats.R[1]),
                        float((ats.lo[2] + l0[2]) * g.h[2] - ats.R[2]), 0.f);
        // the brick's box in the atom's table slot (coordinates of the TMA-staged step)
        tma[((size_t)tl * g.nbricks + br) * g.br_cap + pos_s] = make_int4(tes.atom, l0[0], l0[1], l0[2]);
      }
    }
    cnt += __popc(mask);
  }
  if (lane == 0) {
    bn[(size_t)tl * g.nbricks + br] = min(cnt, g.br_cap);
    if (cnt > g.br_cap) atomicOr(status + kStOverflow, 2);
    if (slab_writer) slab_n[(size_t)tl * g.nslab + by] = srow_base;
  }
}

// A[row][q] = chi_row(x_q) (w_q^T V_nl,q = sum_rows gamma |dOmega| A chi_row^T), the
// projections of t^0 = w_q, Pg0 = gamma |dOmega| A, and a zeroed accumulator Pg1.
template <typename Real>
__global__ void k_atable(Geo g, Wave w, const AtomTab* __restrict__ atoms, const double* __restrict__ chs,
                         const Real* __restrict__ chi, const TileEntry* __restrict__ entries,
                         const int* __restrict__ n_entries, Real* __restrict__ A, double* __restrict__ Pg0_,
                         double* __restrict__ Pg1_) {
  const int tl = blockIdx.x, t = wave_tile(w, tl);
  int o[3];
  tile_origin(g, t, o);
  const int ne = n_entries[tl];
  const TileEntry* ent = entries + (size_t)tl * g.e_cap;
  Real* At = A + (size_t)tl * g.r_cap * g.B;
  double* Pg0 = Pg0_ + (size_t)tl * g.r_cap * g.B;
  double* Pg1 = Pg1_ + (size_t)tl * g.r_cap * g.B;
  for (int i = threadIdx.x; i < ne * g.B; i += blockDim.x) {
    const int e = i / g.B, q = i % g.B;
    const TileEntry te = ent[e];
    const AtomTab at = atoms[te.atom];
    int qo[3];
    node_offset(g, q, qo);
    const bool valid = node_valid(g, o, qo);
    const int li = valid ? box_index(at, te.s, g.n, o[0] + qo[0], o[1] + qo[1], o[2] + qo[2]) : -1;
    const int boxpts = at.dim[0] * at.dim[1] * at.dim[2];
    for (int c = 0; c < at.nch; ++c) {
      const double x = (li >= 0) ? double(chi_row(chi, at, li)[c]) : 0.0;
      At[(size_t)(te.row0 + c) * g.B + q] = Real(x);
      Pg0[(size_t)(te.row0 + c) * g.B + q] = chs[6 * (at.ch0 + c)] * x;   // gamma |dOmega| chi^T t^0
      Pg1[(size_t)(te.row0 + c) * g.B + q] = 0.0;
    }
  }
}

// W_b(u, q) = sum_rows gamma |dOmega| A[row][q] chi_row(u) (x_u,b - R_b) on the window of q:
// contracting the atom sum of the sigma^III term once, S^j_ab = sum_u W_b(u,q) (grad_a t^j)(u).
// One block per (z-plane of bricks, tile); each warp walks whole 4^3 bricks (lanes = 4 x-points x 8
// nodes) and, per half brick (8 points per lane, accumulators in registers), the brick's image
// records: the 64-bit sphere mask skips the points an image does not reach, the table offset
// of the brick corner locates the point's channel group.
template <typename Real>
__global__ void __launch_bounds__(224, sizeof(Real) == 4 ? 4 : 1) k_wtable(Geo g, Wave w, const AtomTab* __restrict__ atoms,
                                                const Real* __restrict__ gdv, const Real* __restrict__ chi,
                                                const TileEntry* __restrict__ entries, const int* __restrict__ blist,
                                                const int4* __restrict__ brec, const float4* __restrict__ bd0,
                                                const int* __restrict__ bn, const Real* __restrict__ A,
                                                Real* __restrict__ W) {
  const int slab = blockIdx.x, tl = blockIdx.y, t = wave_tile(w, tl);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int o[3];
  tile_origin(g, t, o);
  const TileEntry* ent = entries + (size_t)tl * g.e_cap;
  const Real* At = A + (size_t)tl * g.r_cap * g.B;
  Real* Wt = W + (size_t)tl * 3 * g.Upts * g.B;
  const size_t wstr = (size_t)g.Upts * g.B;
  const int q = lane & 7, pa = lane >> 3;
  int qo[3];
  node_offset(g, q, qo);
  const bool valid = node_valid(g, o, qo);
  const Real hr[3] = {Real(g.h[0]), Real(g.h[1]), Real(g.h[2])};
  const int nbx = g.nbr[0], nby = g.nbr[1];
  for (int bi = warp; bi < nbx * nby; bi += nw) {
    const int bx = bi % nbx, by = bi / nbx;
    const int br = (slab * nby + by) * nbx + bx;
    const int4* rb = brec + ((size_t)tl * g.nbricks + br) * g.br_cap * 2;
    const float4* rd = bd0 + ((size_t)tl * g.nbricks + br) * g.br_cap;
    const int* lst = blist + ((size_t)tl * g.nbricks + br) * g.br_cap;
    const int nb = bn[(size_t)tl * g.nbricks + br];
    const int bl[3] = {o[0] - g.m[0] + bx * kBrick, o[1] - g.m[1] + by * kBrick, o[2] - g.m[2] + slab * kBrick};
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      Real acc[8][3];
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = Real(0);
      for (int k = 0; k < nb; ++k) {
        const int4 r0 = rb[2 * k], r1 = rb[2 * k + 1];
        const unsigned mk = unsigned(half ? r1.w : r1.z) >> pa;   // bits pa + 4 i of this half
        if (!(mk & 0x11111111u)) continue;
        // x - R of the brick corner (FP32 path: from the record; FP64: from the image)
        int l0[3] = {0, 0, 0};
        double Ra[3] = {0.0, 0.0, 0.0};
        float4 dc = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (sizeof(Real) == 4) {
          dc = rd[k];
        } else {
          const TileEntry te = ent[lst[k]];
          const AtomTab& at = atoms[te.atom];
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            l0[b] = bl[b] - (at.lo[b] + te.s[b] * g.n[b]);   // box-local lattice coordinates of the corner
            Ra[b] = at.lo[b] * g.h[b] - at.R[b];
          }
        }
        const float dcv[3] = {dc.x, dc.y, dc.z};
        const int nch = r0.w & 0xff, nchp = (r0.w >> 8) & 0xff;
        for (int c0 = 0; c0 < nch; c0 += 4) {
          Real ag[4];
#pragma unroll
          for (int c = 0; c < 4; ++c)
            ag[c] = (c0 + c < nch) ? gdv[r0.z + c0 + c] * At[(size_t)(r0.y + c0 + c) * g.B + q] : Real(0);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if ((mk >> (4 * i)) & 1u) {
              const int it = 8 * half + i, pb = it & 3, pc = it >> 2;
              const Real* cr = chi + r0.x + ((pc * r1.y + pb) * r1.x + pa) * nchp + c0;
              Real cs = Real(0);   // accumulated in the sweep's precision (FP32 suffices for the mixed path)
#pragma unroll
              for (int c = 0; c < 4; ++c) cs += ag[c] * cr[c];
              if (cs == Real(0)) continue;
              const int pt[3] = {pa, pb, pc};
              // x_b - R_b of the image: (l0_b + pt_b) h_b + (lo_b h_b - R_b) (the shift s n h = s L cancels)
#pragma unroll
              for (int b = 0; b < 3; ++b) {
                const Real d = (sizeof(Real) == 4) ? Real(dcv[b]) + Real(pt[b]) * hr[b]
                                                   : Real((l0[b] + pt[b]) * g.h[b] + Ra[b]);
                acc[i][b] += cs * d;
              }
            }
          }
        }
      }
      // the half brick's 8 points of this lane: write W (zero outside the node's window)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int it = 8 * half + i;
        const int ux = bx * kBrick + pa, uy = by * kBrick + (it & 3), uz = slab * kBrick + (it >> 2);
        if (uy >= g.U[1] || uz >= g.U[2]) continue;
        const bool inw = valid && in_window(g, qo, ux, uy, uz);
        const size_t e = ((size_t)(uz * g.U[1] + uy) * g.U[0] + ux) * g.B + q;
#pragma unroll
        for (int b = 0; b < 3; ++b) Wt[b * wstr + e] = inw ? acc[i][b] : Real(0);
      }
    }
  }
}

// t^0 = w_q: one at the node's own point, zero elsewhere (and zero columns for padding nodes).
template <typename Real>
__global__ void k_init_t0(Geo g, Wave w, Real* __restrict__ T0) {
  // T0 was cleared; set t^0 = e_q: 1 at each valid node's own point of the union window
  const int tl = blockIdx.x * blockDim.y + threadIdx.y, q = threadIdx.x;
  if (tl >= w.ntiles) return;
  int o[3], qo[3];
  tile_origin(g, wave_tile(w, tl), o);
  node_offset(g, q, qo);
  if (!node_valid(g, o, qo)) return;
  const int cpt = ((qo[2] + g.m[2]) * g.U[1] + (qo[1] + g.m[1])) * g.U[0] + (qo[0] + g.m[0]);
  T0[((size_t)tl * g.Upts + cpt) * g.B + q] = Real(1);
}

template <typename Real>
static int wave_lists_t(sq_handle* h, const Wave& w, bool reuse, const Real* chi, const Real* gdvR, Real* A, Real* W,
                        Real* T0) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  const sq_handle::ListsKey& key = h->lists_key;
  const bool same = reuse && h->keep_lists && key.full && key.tile0 == w.tile0 && key.ntiles == w.ntiles && key.ids == w.ids &&
                    key.epoch == h->atoms_epoch;
  if (!same) {
    int rc = build_wave_entries(h, w);
    if (rc != SQ_OK) return rc;
  }
  k_atable<Real><<<w.ntiles, 256, 0, s>>>(g, w, h->d.atoms, h->d.gdv, chi, h->wb.entries, h->wb.n_entries, A,
                                          (double*)h->wb.Pg[0], (double*)h->wb.Pg[1]);
  SQ_LAUNCH_CHECK(h);
  if (!same) {
    k_wtable<Real><<<dim3(g.nbr[2], w.ntiles), 224, 0, s>>>(g, w, h->d.atoms, gdvR, chi, h->wb.entries,
                                                            h->wb.brick_list, h->wb.brick_rec, h->wb.brick_d0,
                                                            h->wb.brick_n, A, W);
    SQ_LAUNCH_CHECK(h);
    h->lists_key.full = true;
  }
  SQ_CUDA_TRY(h, cudaMemsetAsync(T0, 0, sizeof(Real) * (size_t)w.ntiles * g.Upts * g.B, s));
  k_init_t0<Real><<<(w.ntiles + 31) / 32, dim3(g.B, 32), 0, s>>>(g, w, T0);
  SQ_LAUNCH_CHECK(h);
  return SQ_OK;
}

int build_wave_entries(sq_handle* h, const Wave& w, WaveBufs* b) {
  const Geo& g = h->geo;
  cudaStream_t s = h->stream;
  if (!b) b = &h->wb;
  if (b == &h->wb) h->lists_key = {w.tile0, w.ntiles, w.ids, h->atoms_epoch, false};
  k_tile_entries<<<w.ntiles, 256, 0, s>>>(g, w, h->d.atoms, b->entries, b->n_entries, b->n_rows, h->d.status);
  SQ_LAUNCH_CHECK(h);
  k_brick_lists<<<dim3(g.nbricks, w.ntiles), 32, 0, s>>>(g, w, h->d.atoms, h->d.rcmax, b->entries, b->n_entries,
                                                          b->brick_list, b->brick_n, b->brick_rec, b->brick_d0,
                                                          b->brick_tma, b->slab_n, b->slab_map, h->d.status);
  SQ_LAUNCH_CHECK(h);
  return SQ_OK;
}

int build_tables(sq_handle* h) {
  if (h->geo.n_atoms == 0 || h->table_len == 0) return SQ_OK;
  k_chi_tables<double><<<h->geo.n_atoms, 256, 0, h->stream>>>(h->geo, h->d.atoms, h->d.gdv, h->d.chi64);
  SQ_LAUNCH_CHECK(h);
  if (h->precision == SQ_MIXED) {
    k_chi_tables<float><<<h->geo.n_atoms, 256, 0, h->stream>>>(h->geo, h->d.atoms, h->d.gdv, h->d.chi32);
    SQ_LAUNCH_CHECK(h);
    k_split_tf32<<<1024, 256, 0, h->stream>>>(h->d.chi32, h->table_len, h->d.chi32s);
    SQ_LAUNCH_CHECK(h);
  }
  return SQ_OK;
}

// cos(pi t / (2 M)) for t in [0, 4 M): cos(j theta_k) = tab[j (2 k + 1) mod 4 M], theta_k = pi (k + 1/2) / M
__global__ void k_costab(int M, double* __restrict__ tab) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 4 * M) tab[t] = cos(M_PI * double(t) / (2.0 * M));
}

// neutral node intervals (0, 1) and zero step coefficients until the per-node Lanczos runs
__global__ void k_node_init(int Nd, double* __restrict__ nbnd, double* __restrict__ ncoef) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Nd) return;
  nbnd[2 * q] = 0.0;
  nbnd[2 * q + 1] = 1.0;
  ncoef[2 * q] = 0.0;
  ncoef[2 * q + 1] = 0.0;
}

int init_node_tables(sq_handle* h) {
  k_costab<<<(4 * h->M + 255) / 256, 256, 0, h->stream>>>(h->M, h->d.costab);
  SQ_LAUNCH_CHECK(h);
  k_node_init<<<(h->Nd + 255) / 256, 256, 0, h->stream>>>(h->Nd, h->d.nbnd, h->d.ncoef);
  SQ_LAUNCH_CHECK(h);
  return SQ_OK;
}

int build_wave_lists(sq_handle* h, const Wave& w, bool reuse) {
  if (h->precision == SQ_FP64)
    return wave_lists_t<double>(h, w, reuse, h->d.chi64, h->d.gdv64, (double*)h->wb.A, (double*)h->wb.W,
                                (double*)h->wb.T[0]);
  return wave_lists_t<float>(h, w, reuse, h->d.chi32, h->d.gdv32, (float*)h->wb.A, (float*)h->wb.W,
                             (float*)h->wb.T[0]);
}

}  // namespace sq
