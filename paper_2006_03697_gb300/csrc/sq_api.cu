// C-ABI entry points and host-side setup of the GB300 SQ library.
//
// The host side validates the descriptor, derives the grid / truncation geometry of Sec. 4
// (h_a, m_a, region of influence), the finite-difference weights of the 2 n_o-order
// central stencils, the per-atom projector support boxes and the tile decomposition; all
// arithmetic of the sweep itself runs in the kernels of sq_setup.cu, sq_sweep.cu and
// sq_reduce.cu.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "sq_internal.h"

namespace {
thread_local std::string g_setup_err = "no error";

long long floor_div(long long a, long long b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

// Central 2 n_o-order finite-difference weights in closed form:
//   second derivative  w_p = 2 (-1)^{p+1} (n_o!)^2 / (p^2 (n_o-p)! (n_o+p)!),  w_0 = -2 sum w_p
//   first derivative   g_p =   (-1)^{p+1} (n_o!)^2 / (p   (n_o-p)! (n_o+p)!)
void fd_weights(int n_o, double* w, double* g) {
  double s = 0.0;
  w[0] = 0.0;
  g[0] = 0.0;
  for (int p = 1; p <= n_o; ++p) {
    // (n_o!)^2 / ((n_o-p)! (n_o+p)!) = prod_{k=1..p} (n_o-p+k) / (n_o+k)
    double base = 1.0;
    for (int k = 1; k <= p; ++k) base *= double(n_o - p + k) / double(n_o + k);
    double sgn = (p % 2 == 1) ? 1.0 : -1.0;
    w[p] = 2.0 * sgn * base / double(p * p);
    g[p] = sgn * base / double(p);
    s += w[p];
  }
  w[0] = -2.0 * s;
}

// Largest number of lattice points of spacing h in an interval of length 2 rc (the support
// box extent of an atom of radius rc on that axis, wherever the atom sits), plus one point of
// slack against rounding in the floor / ceil of place_atom.
int box_extent_max(double rc, double h) { return int(std::floor(2.0 * rc / h + 1e-9)) + 2; }

// An atom's base image (position wrapped into the cell) and its support box for radius rc:
// the lattice points lo_a .. lo_a + dim_a - 1 with |x_a - R_a| <= rc on each axis.
void place_atom(const sq::Geo& g, double rc, const double* pos, sq::AtomTab& at) {
  for (int a = 0; a < 3; ++a) {
    double R = pos[a];
    R -= std::floor(R / g.L[a]) * g.L[a];
    if (R >= g.L[a]) R -= g.L[a];
    at.R[a] = R;
    at.lo[a] = int(std::ceil((R - rc) / g.h[a]));
    const int hi = int(std::floor((R + rc) / g.h[a]));
    // the box keeps the slot's full extent (the points past hi lie outside the sphere and hold
    // zeros), so every table slot of a radius has one shape wherever the atom sits
    (void)hi;
    at.dim[a] = box_extent_max(rc, g.h[a]);
    at.dlo[a] = float(at.lo[a] * g.h[a] - R);
  }
}

int validate(const sq_instance_desc* d, std::string& why) {
  if (!d) { why = "desc is NULL"; return SQ_ERR_INVALID_ARG; }
  for (int a = 0; a < 3; ++a) {
    if (!(d->L[a] > 0.0) || !std::isfinite(d->L[a])) { why = "L must be positive"; return SQ_ERR_INVALID_ARG; }
    if (d->n[a] < 1 || d->n[a] > 4096) { why = "n out of range"; return SQ_ERR_INVALID_ARG; }
  }
  if (d->n_o < 1 || d->n_o > sq::kMaxNo) { why = "n_o must be in [1, 6]"; return SQ_ERR_INVALID_ARG; }
  if (!d->v_eff) { why = "v_eff is NULL"; return SQ_ERR_INVALID_ARG; }
  long long Nd = (long long)d->n[0] * d->n[1] * d->n[2];
  for (long long i = 0; i < Nd; ++i)
    if (!std::isfinite(d->v_eff[i])) { why = "v_eff has a non-finite value"; return SQ_ERR_INVALID_ARG; }
  if (d->n_atoms < 0) { why = "n_atoms < 0"; return SQ_ERR_INVALID_ARG; }
  if (d->n_atoms > 0) {
    if (!d->pos || !d->species || !d->proj_offset || d->n_species < 1) { why = "atom arrays missing"; return SQ_ERR_INVALID_ARG; }
    if (d->proj_offset[0] != 0) { why = "proj_offset[0] must be 0"; return SQ_ERR_INVALID_ARG; }
    for (int s = 0; s < d->n_species; ++s)
      if (d->proj_offset[s + 1] < d->proj_offset[s]) { why = "proj_offset not monotone"; return SQ_ERR_INVALID_ARG; }
    int np = d->proj_offset[d->n_species];
    if (np > 0 && !d->proj) { why = "proj is NULL"; return SQ_ERR_INVALID_ARG; }
    for (int i = 0; i < np; ++i) {
      const sq_proj& p = d->proj[i];
      if (p.l < 0 || p.l > 1) { why = "projector l must be 0 or 1"; return SQ_ERR_INVALID_ARG; }
      if (!(p.width > 0.0) || !std::isfinite(p.gamma)) { why = "projector width/gamma invalid"; return SQ_ERR_INVALID_ARG; }
    }
    for (int J = 0; J < d->n_atoms; ++J) {
      if (d->species[J] < 0 || d->species[J] >= d->n_species) { why = "species index out of range"; return SQ_ERR_INVALID_ARG; }
      int nch = 0;
      for (int i = d->proj_offset[d->species[J]]; i < d->proj_offset[d->species[J] + 1]; ++i) nch += 2 * d->proj[i].l + 1;
      if (nch > sq::kMaxCh) { why = "too many projector channels per atom (max 8)"; return SQ_ERR_INVALID_ARG; }
      for (int a = 0; a < 3; ++a)
        if (!std::isfinite(d->pos[3 * J + a])) { why = "non-finite atom position"; return SQ_ERR_INVALID_ARG; }
    }
  }
  if (!(d->kT > 0.0) || !std::isfinite(d->kT)) { why = "kT must be positive"; return SQ_ERR_INVALID_ARG; }
  if (!(d->n_e > 0.0) || !(d->n_e < 2.0 * double(Nd))) { why = "n_e must be in (0, 2 N_d)"; return SQ_ERR_INVALID_ARG; }
  if (!(d->r_cut > 0.0) || !std::isfinite(d->r_cut)) { why = "r_cut must be positive"; return SQ_ERR_INVALID_ARG; }
  for (int a = 0; a < 3; ++a) {
    int m = int(std::floor(d->r_cut / (d->L[a] / d->n[a]) + 1e-9));
    if (m < 1) { why = "truncation region must contain neighbours (m >= 1)"; return SQ_ERR_INVALID_ARG; }
    if (m > 64) { why = "truncation region too large (m > 64)"; return SQ_ERR_INVALID_ARG; }
  }
  if (d->n_pl < 1 || d->n_pl > 4096) { why = "n_pl out of range"; return SQ_ERR_INVALID_ARG; }
  if (d->lanczos_k > 128) { why = "lanczos_k must be <= 128"; return SQ_ERR_INVALID_ARG; }
  if (d->cheb_quad_M > 6144) { why = "cheb_quad_M must be <= 6144"; return SQ_ERR_INVALID_ARG; }
  if (d->precision != SQ_FP64 && d->precision != SQ_MIXED) { why = "unknown precision"; return SQ_ERR_INVALID_ARG; }
  if (d->bounds_mode != SQ_BOUNDS_LANCZOS && d->bounds_mode != SQ_BOUNDS_GIVEN && d->bounds_mode != SQ_BOUNDS_PER_NODE) {
    why = "unknown bounds mode"; return SQ_ERR_INVALID_ARG;
  }
  if (d->bounds_mode == SQ_BOUNDS_PER_NODE && d->part_count > 0) {
    why = "per-node bounds are not combined with a node partition"; return SQ_ERR_INVALID_ARG;
  }
  if (d->part_count < 0 || (d->part_count > 0 && (d->part_rank < 0 || d->part_rank >= d->part_count))) {
    why = "partition needs 0 <= part_rank < part_count (or part_count = 0)"; return SQ_ERR_INVALID_ARG;
  }
  if (d->bounds_mode == SQ_BOUNDS_GIVEN &&
      !(d->lambda_lo < d->lambda_hi && std::isfinite(d->lambda_lo) && std::isfinite(d->lambda_hi))) {
    why = "given bounds need lambda_lo < lambda_hi"; return SQ_ERR_INVALID_ARG;
  }
  return SQ_OK;
}

// Geometry and buffer sizes shared by sq_setup and sq_footprint_bytes.
struct Plan {
  sq::Geo geo;
  std::vector<sq::AtomTab> atoms;
  std::vector<int> ch_l, ch_m;
  std::vector<double> ch_w, ch_rc, ch_gdv;
  std::vector<double> rcmax;
  long long table_len = 0;
  int wave_cap = 0;
  std::vector<int> lz_tiles;    // sample tiles of the Lanczos bounds
  size_t per_tile_bytes = 0;
  size_t fixed_bytes = 0;
  int tile_begin = 0, tile_end = 0;   // the tiles this handle sweeps (the node partition)
  int lz_cap = 0;                     // most Lanczos sample tiles any V_eff can select
  int nlz_wave = 0;                   // tiles per Lanczos wave of the per-node bounds
};

// Sample nodes of the Lanczos bounds: argmin V, argmax V and a stride-n/2 node grid; their
// tiles, without repeats, in that order.
std::vector<int> lanczos_sample_tiles(const sq::Geo& g, const double* v) {
  const long long Nd = (long long)g.n[0] * g.n[1] * g.n[2];
  std::vector<int> seeds, tiles;
  int imin = 0, imax = 0;
  for (long long i = 1; i < Nd; ++i) {
    if (v[i] < v[imin]) imin = int(i);
    if (v[i] > v[imax]) imax = int(i);
  }
  seeds.push_back(imin);
  seeds.push_back(imax);
  int st[3];
  for (int a = 0; a < 3; ++a) st[a] = std::max(1, g.n[a] / 2);
  for (int iz = 0; iz < g.n[2]; iz += st[2])
    for (int iy = 0; iy < g.n[1]; iy += st[1])
      for (int ix = 0; ix < g.n[0]; ix += st[0]) seeds.push_back(ix + g.n[0] * (iy + g.n[1] * iz));
  for (int q : seeds) {
    const int ix = q % g.n[0], iy = (q / g.n[0]) % g.n[1], iz = q / (g.n[0] * g.n[1]);
    const int t = ix / g.b + g.tiles[0] * (iy / g.b + g.tiles[1] * (iz / g.b));
    if (std::find(tiles.begin(), tiles.end(), t) == tiles.end()) tiles.push_back(t);
  }
  return tiles;
}

int lanczos_sample_cap(const sq::Geo& g) {
  int grid = 1;
  for (int a = 0; a < 3; ++a) {
    const int st = std::max(1, g.n[a] / 2);
    grid *= (g.n[a] + st - 1) / st;
  }
  return std::min(2 + grid, g.n_tiles);
}

int make_plan(const sq_instance_desc* d, Plan& P, std::string& why) {
  sq::Geo& g = P.geo;
  std::memset(&g, 0, sizeof(g));
  g.b = 2;
  g.B = g.b * g.b * g.b;
  g.n_o = d->n_o;
  g.n_pl = d->n_pl;
  g.n_atoms = d->n_atoms;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = d->n[a];
    g.L[a] = d->L[a];
    g.h[a] = d->L[a] / d->n[a];
    g.m[a] = int(std::floor(d->r_cut / g.h[a] + 1e-9));
    g.U[a] = 2 * g.m[a] + g.b;
    if (a == 0) g.U[a] = (g.U[a] + 3) / 4 * 4;   // x extent padded to whole 4-point bricks
    g.nbr[a] = (g.U[a] + sq::kBrick - 1) / sq::kBrick;
    g.tiles[a] = (g.n[a] + g.b - 1) / g.b;
  }
  g.dV = g.h[0] * g.h[1] * g.h[2];
  g.Upts = g.U[0] * g.U[1] * g.U[2];
  g.nbricks = g.nbr[0] * g.nbr[1] * g.nbr[2];
  g.n_tiles = g.tiles[0] * g.tiles[1] * g.tiles[2];
  g.nslab = g.nbr[1];   // slabs are y-rows of bricks (all x, all z)
  double w[sq::kMaxNo + 1], gw[sq::kMaxNo + 1];
  fd_weights(d->n_o, w, gw);
  g.lap0 = 0.0;
  for (int a = 0; a < 3; ++a) {
    g.lap0 += -0.5 * w[0] / (g.h[a] * g.h[a]);
    for (int p = 0; p <= sq::kMaxNo; ++p) {
      g.lap[a][p] = (p <= d->n_o) ? -0.5 * w[p] / (g.h[a] * g.h[a]) : 0.0;
      g.grd[a][p] = (p <= d->n_o) ? gw[p] / g.h[a] : 0.0;
    }
  }
  if (d->precision == SQ_MIXED) {
    // The FP32 sweep multiplies by these weights as floats: store the float values, and pick
    // the centre weight so that the constant mode (exactly 0 for the true stencil) stays as
    // close to 0 as a float allows; the residual is folded into the spectral centre.
    double side = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int p = 1; p <= d->n_o; ++p) {
        g.lap[a][p] = double(float(g.lap[a][p]));
        g.grd[a][p] = double(float(g.grd[a][p]));
        side += 2.0 * g.lap[a][p];
      }
    g.lap0 = double(float(-side));
  }
  g.lap0f = float(g.lap0);
  for (int a = 0; a < 3; ++a)
    for (int p = 0; p <= sq::kMaxNo; ++p) {
      g.lapf[a][p] = float(g.lap[a][p]);
      g.grdf[a][p] = float(g.grd[a][p]);
    }
  // atoms: base image wrapped into the cell, support box of the largest projector radius
  P.atoms.clear();
  long long off = 0;
  int ch = 0;
  long long e_cap = 0, r_cap = 0, br_cap = 0;
  for (int J = 0; J < d->n_atoms; ++J) {
    sq::AtomTab at{};
    std::memset(&at, 0, sizeof(at));
    int s = d->species[J];
    double rc_max = 0.0;
    at.nch = 0;
    at.ch0 = ch;
    for (int i = d->proj_offset[s]; i < d->proj_offset[s + 1]; ++i) {
      const sq_proj& p = d->proj[i];
      double rc = (p.rcut > 0.0) ? p.rcut : 7.0 * p.width;
      rc_max = std::max(rc_max, rc);
      for (int mch = 0; mch < 2 * p.l + 1; ++mch) {
        P.ch_l.push_back(p.l);
        P.ch_m.push_back(mch);
        P.ch_w.push_back(p.width);
        P.ch_rc.push_back(rc);
        P.ch_gdv.push_back(p.gamma * g.dV);
        at.nch++;
        ch++;
      }
    }
    place_atom(g, rc_max, d->pos + 3 * J, at);
    // every atom owns a fixed table slot sized for the largest support box its radius allows
    // anywhere in the cell, so a handle can take new positions in place (sq_update_atoms)
    int dmax[3];
    long long slot = 1;
    for (int a = 0; a < 3; ++a) {
      dmax[a] = box_extent_max(rc_max, g.h[a]);
      slot *= dmax[a];
    }
    if (at.nch == 0) slot = 0;
    P.rcmax.push_back(rc_max);
    at.nchp = (at.nch + 3) / 4 * 4;
    at.off = off;
    off += slot * at.nchp;
    // capacity bounds: images of this atom that can meet a window of extent W on axis a
    long long nimg_u = 1, nimg_b = 1;
    for (int a = 0; a < 3; ++a) {
      nimg_u *= floor_div(g.U[a] + dmax[a] - 2, g.n[a]) + 1;
      nimg_b *= floor_div(sq::kBrick + dmax[a] - 2, g.n[a]) + 1;
    }
    if (at.nch == 0) { nimg_u = nimg_b = 0; }
    e_cap += nimg_u;
    r_cap += nimg_u * at.nch;
    br_cap += nimg_b;
    P.atoms.push_back(at);
  }
  P.table_len = off;
  if (off >= (1ll << 31)) { why = "projector tables exceed 2^31 entries"; return SQ_ERR_INVALID_ARG; }
  g.e_cap = int(std::max<long long>(1, std::min<long long>(e_cap, 1 << 20)));
  g.r_cap = int(std::max<long long>(1, std::min<long long>(r_cap, 1 << 22)));
  g.br_cap = int(std::max<long long>(1, std::min<long long>(br_cap, g.e_cap)));
  if (e_cap > (1 << 20) || r_cap > (1 << 22)) { why = "too many atom images per tile"; return SQ_ERR_INVALID_ARG; }

  size_t real = (d->precision == SQ_FP64) ? sizeof(double) : sizeof(float);
  size_t tileB = size_t(g.B);
  P.per_tile_bytes = size_t(g.e_cap) * sizeof(sq::TileEntry) + 2 * sizeof(int) +
                     size_t(g.nbricks) * (size_t(g.br_cap) + 1) * sizeof(int) +
                     size_t(g.nbricks) * size_t(g.br_cap) * 4 * sizeof(int4) +   // records, corner offsets, TMA boxes
                     3 * size_t(g.Upts) * tileB * real +        // T ring
                     3 * size_t(g.Upts) * tileB * real +        // W
                     2 * size_t(g.r_cap) * tileB * real +       // A, P
                     2 * size_t(g.r_cap) * tileB * sizeof(double) +   // Pg ping-pong (FP64)
                     size_t(g.nslab) * tileB * 9 * sizeof(double) +
                     size_t(g.nslab) * (size_t(g.r_cap) + 1) * sizeof(int);   // slab row maps
  long long Nd = (long long)g.n[0] * g.n[1] * g.n[2];
  int M = d->cheb_quad_M > 0 ? d->cheb_quad_M : 2048;
  P.fixed_bytes = size_t(Nd) * (sizeof(double) + sizeof(float)) +                       // V
                  P.atoms.size() * sizeof(sq::AtomTab) + size_t(ch) * 6 * sizeof(double) +
                  // projector tables: FP64 (always; the Lanczos apply and the FP64 sweep), FP32 and
                  // TF32 hi/lo pairs for the mixed sweep
                  size_t(P.table_len) * (sizeof(double) + (real == sizeof(float) ? 3 * sizeof(float) : 0)) +
                  size_t(Nd) * size_t(d->n_pl + 1) * SQ_N_MOMENTS * sizeof(double) +   // moments
                  size_t(d->n_pl + 1) * 4 * sizeof(double) + size_t(M) * sizeof(double) +
                  size_t(Nd) * sizeof(double) + 4096 * 32 * sizeof(double) + sq::kLzDotCap * sizeof(double) + 1024;
  // Lanczos sample tiles (argmin V, argmax V, a stride-n/2 node grid); the buffers hold the
  // largest count so that sq_update_atoms can move them with V
  P.lz_tiles.clear();
  if (d->bounds_mode == SQ_BOUNDS_LANCZOS) {
    P.lz_tiles = lanczos_sample_tiles(g, d->v_eff);
    P.lz_cap = lanczos_sample_cap(g);
    const int k = d->lanczos_k > 0 ? d->lanczos_k : 40;
    const size_t nst = size_t(P.lz_cap);
    P.fixed_bytes += sizeof(double) * (size_t(k + 2) * nst * g.Upts * g.B + nst * size_t(g.r_cap) * g.B +
                                       nst * g.B * size_t(5 * k + 8)) + sizeof(int) * nst;
    // the sample tiles' own entry and brick lists
    P.fixed_bytes += nst * (size_t(g.e_cap) * sizeof(sq::TileEntry) + 2 * sizeof(int) +
                            size_t(g.nbricks) * (size_t(g.br_cap) + 1) * sizeof(int) +
                            size_t(g.nbricks) * size_t(g.br_cap) * 4 * sizeof(int4) +
                            size_t(g.nslab) * (size_t(g.r_cap) + 1) * sizeof(int));
  }
  // the node partition: part part_rank of part_count equal contiguous tile ranges
  P.tile_begin = 0;
  P.tile_end = g.n_tiles;
  if (d->part_count > 0) {
    P.tile_begin = int((long long)g.n_tiles * d->part_rank / d->part_count);
    P.tile_end = int((long long)g.n_tiles * (d->part_rank + 1) / d->part_count);
  }
  const long long ntl = std::max(1, P.tile_end - P.tile_begin);
  // tiles per wave: one wave when the whole working set fits in 64 GiB (its lists and W table are
  // then built once and kept across evaluations), else waves of at most 24 GiB (fewer, larger
  // launches: less per-wave setup and a smaller tail), with the tiles spread evenly over the waves
  size_t budget = size_t(24) << 30;
  if (size_t(ntl) * P.per_tile_bytes <= (size_t(64) << 30)) budget = size_t(ntl) * P.per_tile_bytes;
  long long wc = std::max<long long>(1, (long long)(budget / std::max<size_t>(P.per_tile_bytes, 1)));
  wc = std::min<long long>(std::min<long long>(wc, ntl), 32768);
  const long long nwaves = (ntl + wc - 1) / wc;
  P.wave_cap = int((ntl + nwaves - 1) / nwaves);
  P.wave_cap = std::max<int>(P.wave_cap, P.lz_cap);
  if (d->bounds_mode == SQ_BOUNDS_PER_NODE) {
    // every node's own Lanczos: waves of tiles with k + 2 Krylov vectors each under 8 GiB, the
    // per-node interval and step coefficients, the Fermi-search cosine sums and contraction rows
    const int k = d->lanczos_k > 0 ? d->lanczos_k : 40;
    const size_t per_tile = (size_t(k + 2) * g.Upts + size_t(g.r_cap)) * g.B * real + size_t(g.B) * (5 * k + 8) * 8;
    P.nlz_wave = int(std::max<size_t>(1, std::min<size_t>((size_t(8) << 30) / per_tile, size_t(P.wave_cap))));
    P.fixed_bytes += size_t(P.nlz_wave) * per_tile + size_t(Nd) * (4 + M + 20) * sizeof(double) +
                     size_t(4 * M + 1024) * sizeof(double);
  }
  return SQ_OK;
}
}  // namespace

namespace sq {

int fail(sq_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_setup_err = msg;
  return code;
}

// Given bounds go through the same device scaling as the Lanczos ones (set_bounds_device):
// the FP32-exact coefficients of SQ_MIXED, one rounding of the diagonal coefficient, and the
// effective interval the recurrence realises.
int set_bounds(sq_handle* h, double lo, double hi) {
  h->hscal[0] = lo;
  h->hscal[1] = hi;
  cudaError_t e = cudaMemcpyAsync(h->d.scal + 8, h->hscal, 2 * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return fail(h, SQ_ERR_CUDA, std::string("set_bounds: ") + cudaGetErrorString(e));
  return set_bounds_device(h);
}

cudaEvent_t timing_begin(sq_handle* h, int kid, double bytes) {
  if (!h->timing) return nullptr;
  const size_t need = 2 * (h->ev_pending.size() + 1);
  while (h->ev_pool.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev_pool.push_back(e);
  }
  cudaEvent_t e0 = h->ev_pool[2 * h->ev_pending.size()];
  h->ev_pending.push_back({kid, bytes});
  cudaEventRecord(e0, h->stream);
  return e0;
}

void timing_end(sq_handle* h, cudaEvent_t start) {
  if (!start) return;
  cudaEventRecord(h->ev_pool[2 * h->ev_pending.size() - 1], h->stream);
}

int timing_collect(sq_handle* h) {
  if (h->ev_pending.empty()) return SQ_OK;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, SQ_ERR_CUDA, std::string("timing sync: ") + cudaGetErrorString(e));
  for (size_t i = 0; i < h->ev_pending.size(); ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]) == cudaSuccess) {
      const int kid = h->ev_pending[i].first;
      h->t_launches[kid] += 1;
      h->t_ms[kid] += ms;
      h->t_bytes[kid] += h->ev_pending[i].second;
    }
  }
  h->ev_pending.clear();
  return SQ_OK;
}

int dev_alloc(sq_handle* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(h, SQ_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  h->allocs.push_back(*p);
  h->bytes += bytes;
  return SQ_OK;
}

}  // namespace sq

extern "C" {

size_t sq_footprint_bytes(const sq_instance_desc* desc) {
  std::string why;
  if (validate(desc, why) != SQ_OK) return 0;
  Plan P;
  if (make_plan(desc, P, why) != SQ_OK) return 0;
  return P.fixed_bytes + size_t(P.wave_cap) * P.per_tile_bytes;
}

int sq_setup(const sq_instance_desc* desc, sq_handle** out) {
  sq::NvtxRange nvtx("sq_setup");
  if (!out) { g_setup_err = "out is NULL"; return SQ_ERR_INVALID_ARG; }
  *out = nullptr;
  std::string why;
  int rc = validate(desc, why);
  if (rc != SQ_OK) { g_setup_err = why; return rc; }
  Plan P;
  rc = make_plan(desc, P, why);
  if (rc != SQ_OK) { g_setup_err = why; return rc; }

  sq_handle* h = new sq_handle();
  h->desc = *desc;
  h->desc.v_eff = nullptr;
  h->desc.pos = nullptr;
  h->desc.species = nullptr;
  h->desc.proj_offset = nullptr;
  h->desc.proj = nullptr;
  h->geo = P.geo;
  h->precision = desc->precision;
  h->bounds_mode = desc->bounds_mode;
  h->M = desc->cheb_quad_M > 0 ? desc->cheb_quad_M : 2048;
  h->lanczos_k = desc->lanczos_k > 0 ? desc->lanczos_k : 40;
  h->kT = desc->kT;
  h->n_e = desc->n_e;
  h->Nd = desc->n[0] * desc->n[1] * desc->n[2];
  h->vol = desc->L[0] * desc->L[1] * desc->L[2];
  h->stream = (cudaStream_t)desc->stream;
  h->atoms_h = P.atoms;
  h->rcmax_h = P.rcmax;
  h->lz_cap = P.lz_cap;
  h->nlz_wave = P.nlz_wave;
  h->proj4 = true;
  for (const sq::AtomTab& at : P.atoms) h->proj4 = h->proj4 && at.nchp <= 4;
  h->table_len = P.table_len;
  h->n_ch_total = int(P.ch_l.size());
  h->wave_cap = P.wave_cap;
  for (int t0 = P.tile_begin; t0 < P.tile_end; t0 += h->wave_cap)
    h->waves.push_back({t0, std::min(h->wave_cap, P.tile_end - t0), nullptr});
  h->tile_begin = P.tile_begin;
  h->tile_end = P.tile_end;
  h->lanczos_tiles = P.lz_tiles;
  // projector rows a step block may stage in shared memory; SQ_STEP_SMEM_ROWS lowers the cap
  // (tuning and tests of the global-memory projection path)
  h->step_rows_cap = sq::step_rows_smem_max(desc->precision);
  if (const char* env = std::getenv("SQ_STEP_SMEM_ROWS")) {
    const long v = std::strtol(env, nullptr, 10);
    if (v >= 0 && v < h->step_rows_cap) h->step_rows_cap = int(v);
  }
  // SQ_STEP_KERNEL=staged selects the TMA-staged step for a mixed sweep (sq_step_tma.cu; slower than
  // the default step kernel on the workloads measured, kept for comparison), SQ_STAGE_RECS its
  // images per stage
  if (const char* env = std::getenv("SQ_STEP_KERNEL")) h->step_staged = std::string(env) == "staged";
  // SQ_STAGE_WAIT_TEST=1: every stage of the staged step waits for 16 bytes that never come, so
  // its bounded wait runs out (the test of SQ_ERR_TIMEOUT; the copies themselves complete)
  if (const char* env = std::getenv("SQ_STAGE_WAIT_TEST")) h->stage_wait_test = std::string(env) == "1";
  if (const char* env = std::getenv("SQ_STAGE_RECS")) {
    const long v = std::strtol(env, nullptr, 10);
    if (v >= 1 && v <= 64) h->stage_recs_cap = int(v);
  }

  auto cleanup = [&](int code) {
    g_setup_err = h->err;
    sq_destroy(h);
    return code;
  };
  const bool f64 = h->precision == SQ_FP64;
  const size_t real = f64 ? sizeof(double) : sizeof(float);
  const sq::Geo& g = h->geo;
  const int Nd = h->Nd;
  void* p = nullptr;
#define SQ_ALLOC(field, bytes)                                   \
  do {                                                           \
    int rc_ = sq::dev_alloc(h, &p, (bytes));                     \
    if (rc_ != SQ_OK) return cleanup(rc_);                       \
    field = decltype(field)(p);                                  \
  } while (0)
  SQ_ALLOC(h->d.v64, sizeof(double) * Nd);
  SQ_ALLOC(h->d.v32, sizeof(float) * Nd);
  SQ_ALLOC(h->d.atoms, sizeof(sq::AtomTab) * std::max<size_t>(1, P.atoms.size()));
  SQ_ALLOC(h->d.gdv, sizeof(double) * std::max(1, h->n_ch_total) * 6);
  SQ_ALLOC(h->d.gdv64, sizeof(double) * std::max(1, h->n_ch_total));
  SQ_ALLOC(h->d.rcmax, sizeof(double) * std::max<size_t>(1, P.rcmax.size()));
  SQ_ALLOC(h->d.gdv32, sizeof(float) * std::max(1, h->n_ch_total));
  SQ_ALLOC(h->d.chi64, sizeof(double) * std::max<long long>(1, P.table_len));
  if (!f64) SQ_ALLOC(h->d.chi32, sizeof(float) * std::max<long long>(1, P.table_len));
  if (!f64) SQ_ALLOC(h->d.chi32s, 2 * sizeof(float) * std::max<long long>(1, P.table_len));
  SQ_ALLOC(h->d.mom, sizeof(double) * size_t(Nd) * size_t(g.n_pl + 1) * SQ_N_MOMENTS);
  SQ_ALLOC(h->d.R, sizeof(double) * (g.n_pl + 1));
  SQ_ALLOC(h->d.cosF, sizeof(double) * h->M);
  SQ_ALLOC(h->d.coef, sizeof(double) * 3 * (g.n_pl + 1));
  SQ_ALLOC(h->d.scal, sizeof(double) * 64);
  SQ_ALLOC(h->d.part, sizeof(double) * 4096 * 32);
  SQ_ALLOC(h->d.rho, sizeof(double) * Nd);
  SQ_ALLOC(h->d.status, sizeof(int) * sq::kStCount);
  SQ_ALLOC(h->d.lzdot, sizeof(double) * sq::kLzDotCap);
  const int wt = h->wave_cap;
  SQ_ALLOC(h->wb.entries, sizeof(sq::TileEntry) * size_t(wt) * g.e_cap);
  SQ_ALLOC(h->wb.n_entries, sizeof(int) * wt);
  SQ_ALLOC(h->wb.n_rows, sizeof(int) * wt);
  SQ_ALLOC(h->wb.brick_list, sizeof(int) * size_t(wt) * g.nbricks * g.br_cap);
  SQ_ALLOC(h->wb.brick_n, sizeof(int) * size_t(wt) * g.nbricks);
  SQ_ALLOC(h->wb.brick_rec, sizeof(int4) * 2 * size_t(wt) * g.nbricks * g.br_cap);
  SQ_ALLOC(h->wb.brick_d0, sizeof(float4) * size_t(wt) * g.nbricks * g.br_cap);
  SQ_ALLOC(h->wb.brick_tma, sizeof(int4) * size_t(wt) * g.nbricks * g.br_cap);
  SQ_ALLOC(h->wb.slab_n, sizeof(int) * size_t(wt) * g.nslab);
  SQ_ALLOC(h->wb.slab_map, sizeof(int) * size_t(wt) * g.nslab * g.r_cap);
  for (int i = 0; i < 3; ++i) SQ_ALLOC(h->wb.T[i], real * size_t(wt) * g.Upts * g.B);
  SQ_ALLOC(h->wb.W, real * size_t(wt) * 3 * g.Upts * g.B);
  SQ_ALLOC(h->wb.A, real * size_t(wt) * g.r_cap * g.B);
  SQ_ALLOC(h->wb.P, real * size_t(wt) * g.r_cap * g.B);
  SQ_ALLOC(h->wb.Pg[0], sizeof(double) * size_t(wt) * g.r_cap * g.B);   // projections: FP64 sums
  SQ_ALLOC(h->wb.Pg[1], sizeof(double) * size_t(wt) * g.r_cap * g.B);
  SQ_ALLOC(h->wb.Spart, sizeof(double) * size_t(wt) * g.nslab * g.B * 9);
  if (!h->lanczos_tiles.empty()) {
    const size_t nst = size_t(P.lz_cap);
    const int k = h->lanczos_k;
    SQ_ALLOC(h->d.lzV, sizeof(double) * size_t(k + 1) * nst * g.Upts * g.B);
    SQ_ALLOC(h->d.lzW, sizeof(double) * nst * g.Upts * g.B);
    SQ_ALLOC(h->d.lzP, sizeof(double) * nst * size_t(g.r_cap) * g.B);
    SQ_ALLOC(h->d.lzC, sizeof(double) * nst * g.B * size_t(5 * k + 8));
    SQ_ALLOC(h->d.lz_tiles, sizeof(int) * nst);
    // list buffers of the sample tiles (the sweep's wave lists stay untouched by the bounds)
    SQ_ALLOC(h->lzb.entries, sizeof(sq::TileEntry) * nst * g.e_cap);
    SQ_ALLOC(h->lzb.n_entries, sizeof(int) * nst);
    SQ_ALLOC(h->lzb.n_rows, sizeof(int) * nst);
    SQ_ALLOC(h->lzb.brick_list, sizeof(int) * nst * g.nbricks * g.br_cap);
    SQ_ALLOC(h->lzb.brick_n, sizeof(int) * nst * g.nbricks);
    SQ_ALLOC(h->lzb.brick_rec, sizeof(int4) * 2 * nst * g.nbricks * g.br_cap);
    SQ_ALLOC(h->lzb.brick_d0, sizeof(float4) * nst * g.nbricks * g.br_cap);
    SQ_ALLOC(h->lzb.brick_tma, sizeof(int4) * nst * g.nbricks * g.br_cap);
    SQ_ALLOC(h->lzb.slab_n, sizeof(int) * nst * g.nslab);
    SQ_ALLOC(h->lzb.slab_map, sizeof(int) * nst * g.nslab * g.r_cap);
  }
  if (h->bounds_mode == SQ_BOUNDS_PER_NODE) {
    const int k = h->lanczos_k;
    const size_t nw = size_t(h->nlz_wave);
    SQ_ALLOC(h->d.nbnd, sizeof(double) * 2 * size_t(Nd));
    SQ_ALLOC(h->d.ncoef, sizeof(double) * 2 * size_t(Nd));
    SQ_ALLOC(h->d.nF, sizeof(double) * size_t(Nd) * h->M);
    SQ_ALLOC(h->d.nrow, sizeof(double) * size_t(Nd) * 20);
    SQ_ALLOC(h->d.costab, sizeof(double) * 4 * size_t(h->M));
    SQ_ALLOC(h->d.npart, sizeof(double) * 1024);
    SQ_ALLOC(h->d.nV, real * size_t(k + 1) * nw * g.Upts * g.B);
    SQ_ALLOC(h->d.nW, real * nw * g.Upts * g.B);
    SQ_ALLOC(h->d.nP, real * nw * size_t(g.r_cap) * g.B);
    SQ_ALLOC(h->d.nC, sizeof(double) * nw * g.B * size_t(5 * k + 8));
  }
#undef SQ_ALLOC

  // inputs -> device
  std::vector<float> v32(Nd);
  for (int i = 0; i < Nd; ++i) v32[i] = float(desc->v_eff[i]);
  std::vector<double> chs(size_t(std::max(1, h->n_ch_total)) * 6, 0.0);
  for (int c = 0; c < h->n_ch_total; ++c) {
    chs[6 * c + 0] = P.ch_gdv[c];
    chs[6 * c + 1] = double(P.ch_l[c]);
    chs[6 * c + 2] = double(P.ch_m[c]);
    chs[6 * c + 3] = P.ch_w[c];
    chs[6 * c + 4] = P.ch_rc[c];
  }
  cudaStream_t s = h->stream;
#define SQ_H2D(dst, src, bytes)                                                          \
  do {                                                                                   \
    cudaError_t e_ = cudaMemcpyAsync((dst), (src), (bytes), cudaMemcpyHostToDevice, s); \
    if (e_ != cudaSuccess) {                                                             \
      sq::fail(h, SQ_ERR_CUDA, std::string("H2D: ") + cudaGetErrorString(e_));           \
      return cleanup(SQ_ERR_CUDA);                                                       \
    }                                                                                    \
  } while (0)
  SQ_H2D(h->d.v64, desc->v_eff, sizeof(double) * Nd);
  SQ_H2D(h->d.v32, v32.data(), sizeof(float) * Nd);
  if (!P.atoms.empty()) SQ_H2D(h->d.atoms, P.atoms.data(), sizeof(sq::AtomTab) * P.atoms.size());
  SQ_H2D(h->d.gdv, chs.data(), sizeof(double) * chs.size());
  std::vector<double> g64(std::max(1, h->n_ch_total), 0.0);
  std::vector<float> g32(std::max(1, h->n_ch_total), 0.f);
  for (int c = 0; c < h->n_ch_total; ++c) {
    g64[c] = P.ch_gdv[c];
    g32[c] = float(P.ch_gdv[c]);
  }
  SQ_H2D(h->d.gdv64, g64.data(), sizeof(double) * g64.size());
  if (!P.rcmax.empty()) SQ_H2D(h->d.rcmax, P.rcmax.data(), sizeof(double) * P.rcmax.size());
  SQ_H2D(h->d.gdv32, g32.data(), sizeof(float) * g32.size());
  if (!h->lanczos_tiles.empty())
    SQ_H2D(h->d.lz_tiles, h->lanczos_tiles.data(), sizeof(int) * h->lanczos_tiles.size());
  double sc[64];
  std::memset(sc, 0, sizeof(sc));
  SQ_H2D(h->d.scal, sc, sizeof(sc));
  {
    double side = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int p = 1; p <= g.n_o; ++p) side += 2.0 * g.lap[a][p];
    h->lap_offset = g.lap0 + side;
  }
  if (h->bounds_mode == SQ_BOUNDS_GIVEN) {
    rc = sq::set_bounds(h, desc->lambda_lo, desc->lambda_hi);
    if (rc != SQ_OK) return cleanup(rc);
    h->bounds_ready = true;
  }
#undef SQ_H2D
  if (cudaMemsetAsync(h->d.mom, 0, sizeof(double) * size_t(Nd) * size_t(g.n_pl + 1) * SQ_N_MOMENTS, s) !=
      cudaSuccess) {
    sq::fail(h, SQ_ERR_CUDA, "memset moments");
    return cleanup(SQ_ERR_CUDA);
  }
  if (cudaMemsetAsync(h->d.status, 0, sizeof(int) * sq::kStCount, s) != cudaSuccess) {
    sq::fail(h, SQ_ERR_CUDA, "memset status");
    return cleanup(SQ_ERR_CUDA);
  }
  rc = sq::build_tables(h);
  if (rc != SQ_OK) return cleanup(rc);
  rc = sq::make_step_maps(h);
  if (rc != SQ_OK) return cleanup(rc);
  if (h->bounds_mode == SQ_BOUNDS_PER_NODE) {
    rc = sq::init_node_tables(h);
    if (rc != SQ_OK) return cleanup(rc);
  }
  rc = sq::measure_wave_rows(h);   // the sweep then needs no host round trip
  if (rc != SQ_OK) return cleanup(rc);

  *out = h;
  return SQ_OK;
}

int sq_moments(sq_handle* h) {
  if (!h) return SQ_ERR_INVALID_ARG;
  sq::NvtxRange nvtx("sq_moments");
  int rc;
  if (h->bounds_mode == SQ_BOUNDS_LANCZOS) {   // bounds are part of every sweep
    sq::NvtxRange nb("bounds: Lanczos");
    rc = sq::run_lanczos(h);
    if (rc != SQ_OK) return rc;
    h->bounds_ready = true;
  } else if (h->bounds_mode == SQ_BOUNDS_PER_NODE) {
    sq::NvtxRange nb("bounds: per-node Lanczos");
    rc = sq::run_lanczos_nodes(h);
    if (rc != SQ_OK) return rc;
    h->bounds_ready = true;
  }
  rc = sq::run_sweep(h);
  if (rc != SQ_OK) return rc;
  h->moments_ready = true;
  return SQ_OK;
}

int sq_fermi_level(sq_handle* h, double* mu_out) {
  if (!h) return SQ_ERR_INVALID_ARG;
  if (!h->moments_ready) return sq::fail(h, SQ_ERR_STATE, "sq_fermi_level before sq_moments");
  sq::NvtxRange nvtx("sq_fermi_level");
  if (h->bounds_mode == SQ_BOUNDS_PER_NODE) return sq::run_fermi_nodes(h, mu_out);
  return sq::run_fermi(h, mu_out);
}

int sq_update_atoms(sq_handle* h, const double* pos, const double* v_eff) {
  if (!h) return SQ_ERR_INVALID_ARG;
  sq::NvtxRange nvtx("sq_update_atoms");
  const sq::Geo& g = h->geo;
  if (!v_eff || (g.n_atoms > 0 && !pos)) return sq::fail(h, SQ_ERR_INVALID_ARG, "pos or v_eff is NULL");
  for (int i = 0; i < h->Nd; ++i)
    if (!std::isfinite(v_eff[i])) return sq::fail(h, SQ_ERR_INVALID_ARG, "v_eff has a non-finite value");
  for (int i = 0; i < 3 * g.n_atoms; ++i)
    if (!std::isfinite(pos[i])) return sq::fail(h, SQ_ERR_INVALID_ARG, "non-finite atom position");
  // new base images and support boxes inside each atom's fixed table slot
  bool moved = false;
  for (int J = 0; J < g.n_atoms; ++J) {
    const double R0[3] = {h->atoms_h[J].R[0], h->atoms_h[J].R[1], h->atoms_h[J].R[2]};
    place_atom(g, h->rcmax_h[J], pos + 3 * J, h->atoms_h[J]);
    for (int a = 0; a < 3; ++a) moved = moved || h->atoms_h[J].R[a] != R0[a];
  }
  if (moved) h->atoms_epoch++;   // kept wave lists and W table describe the old positions
  cudaStream_t s = h->stream;
  std::vector<float> v32(h->Nd);
  for (int i = 0; i < h->Nd; ++i) v32[i] = float(v_eff[i]);
  SQ_CUDA_TRY(h, cudaMemcpyAsync(h->d.v64, v_eff, sizeof(double) * h->Nd, cudaMemcpyHostToDevice, s));
  SQ_CUDA_TRY(h, cudaMemcpyAsync(h->d.v32, v32.data(), sizeof(float) * h->Nd, cudaMemcpyHostToDevice, s));
  if (g.n_atoms > 0)
    SQ_CUDA_TRY(h, cudaMemcpyAsync(h->d.atoms, h->atoms_h.data(), sizeof(sq::AtomTab) * h->atoms_h.size(),
                                   cudaMemcpyHostToDevice, s));
  if (h->bounds_mode == SQ_BOUNDS_LANCZOS) {
    // the sample tiles follow argmin / argmax of the new V_eff
    std::vector<int> lz = lanczos_sample_tiles(g, v_eff);
    if (int(lz.size()) > h->lz_cap) return sq::fail(h, SQ_ERR_STATE, "Lanczos sample capacity exceeded");
    if (lz != h->lanczos_tiles) h->lz_lists_epoch = -1;   // other sample tiles: their lists are rebuilt
    h->lanczos_tiles = lz;
    SQ_CUDA_TRY(h, cudaMemcpyAsync(h->d.lz_tiles, lz.data(), sizeof(int) * lz.size(), cudaMemcpyHostToDevice, s));
    h->bounds_ready = false;
  }
  int rc = sq::build_tables(h);
  if (rc != SQ_OK) return rc;
  if (moved) {
    rc = sq::measure_wave_rows(h);   // the atoms moved: the slabs meet other projector rows
    if (rc != SQ_OK) return rc;
  }
  // pageable host sources: the copies have read them before the call returns; the handle's
  // results now describe the new snapshot only after the next sq_moments
  SQ_CUDA_TRY(h, cudaStreamSynchronize(s));
  h->moments_ready = false;
  return SQ_OK;
}

int sq_node_sums(sq_handle* h, double* R_out) {
  if (!h || !R_out) return SQ_ERR_INVALID_ARG;
  if (!h->moments_ready) return sq::fail(h, SQ_ERR_STATE, "sq_node_sums before sq_moments");
  return sq::run_node_sums(h, R_out);
}

int sq_fermi_level_sums(sq_handle* h, const double* R_host, double* mu_out) {
  if (!h) return SQ_ERR_INVALID_ARG;
  if (!R_host) return sq::fail(h, SQ_ERR_INVALID_ARG, "R_host is NULL");
  for (int j = 0; j <= h->geo.n_pl; ++j)
    if (!std::isfinite(R_host[j])) return sq::fail(h, SQ_ERR_INVALID_ARG, "R_host has a non-finite value");
  if (!h->bounds_ready) return sq::fail(h, SQ_ERR_STATE, "sq_fermi_level_sums before the bounds are known");
  if (h->bounds_mode == SQ_BOUNDS_PER_NODE)
    return sq::fail(h, SQ_ERR_STATE, "node sums carry no per-node coefficients (SQ_BOUNDS_PER_NODE)");
  return sq::run_fermi_sums(h, R_host, mu_out);
}

static int contraction_common(sq_handle* h, double mu, double* rho_dev, sq_energies* e_out,
                              double* sigma_host, double* sigma_dev, double* pressure_host = nullptr) {
  if (!h) return SQ_ERR_INVALID_ARG;
  if (!h->moments_ready) return sq::fail(h, SQ_ERR_STATE, "contraction before sq_moments");
  if (!std::isfinite(mu)) return sq::fail(h, SQ_ERR_INVALID_ARG, "mu is not finite");
  sq::NvtxRange nvtx("contraction");
  double out[16];
  double* sums = (e_out || sigma_host || pressure_host) ? out : nullptr;
  int rc = (h->bounds_mode == SQ_BOUNDS_PER_NODE) ? sq::run_contraction_nodes(h, mu, rho_dev, sums)
                                                  : sq::run_contraction(h, mu, rho_dev, sums);
  if (rc != SQ_OK) return rc;
  if (pressure_host) {
    pressure_host[0] = out[14];
    pressure_host[1] = out[13];
  }
  if (e_out) {
    e_out->E_band = out[0];
    e_out->E_s = out[1];
    e_out->E_nl = out[2];
    e_out->F = out[0] + out[1];
    e_out->N_check = out[3];
    e_out->mu = mu;
  }
  if (sigma_host) std::memcpy(sigma_host, out + 4, 9 * sizeof(double));
  if (sigma_dev) {
    SQ_CUDA_TRY(h, cudaMemcpyAsync(sigma_dev, h->d.scal + 20, 9 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  }
  return SQ_OK;
}

int sq_density_energy_stress(sq_handle* h, double mu, double* rho_out, sq_energies* e_out, double* sigma_out) {
  if (!h) return SQ_ERR_INVALID_ARG;
  int rc = contraction_common(h, mu, h->d.rho, e_out, sigma_out, nullptr);
  if (rc != SQ_OK) return rc;
  if (rho_out) {
    SQ_CUDA_TRY(h, cudaMemcpyAsync(rho_out, h->d.rho, sizeof(double) * h->Nd, cudaMemcpyDeviceToHost, h->stream));
    SQ_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return SQ_OK;
}

int sq_density_energy_stress_dev(sq_handle* h, double mu, double* rho_dev, sq_energies* e_out, double* sigma_dev) {
  if (!h) return SQ_ERR_INVALID_ARG;
  return contraction_common(h, mu, rho_dev ? rho_dev : h->d.rho, e_out, nullptr, sigma_dev);
}

int sq_pressure(sq_handle* h, double mu, double* pressure_out, double* e_pot_out) {
  if (!h || !pressure_out) return SQ_ERR_INVALID_ARG;
  double pe[2];
  int rc = contraction_common(h, mu, h->d.rho, nullptr, nullptr, nullptr, pe);
  if (rc != SQ_OK) return rc;
  *pressure_out = pe[0];
  if (e_pot_out) *e_pot_out = pe[1];
  return SQ_OK;
}

int sq_get_bounds(const sq_handle* h, double* lo, double* hi) {
  if (!h || !lo || !hi) return SQ_ERR_INVALID_ARG;
  if (!h->bounds_ready) return SQ_ERR_STATE;
  if (h->bounds_mode == SQ_BOUNDS_PER_NODE) {
    *lo = h->lam_lo;
    *hi = h->lam_hi;
    return SQ_OK;
  }
  // the effective interval lives on the device (scaled there, from the Lanczos or given bounds)
  double b[2];
  int st[sq::kStCount];
  if (cudaMemcpyAsync(b, h->d.scal, sizeof(b), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(st, h->d.status, sizeof(st), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return SQ_ERR_CUDA;
  }
  if (st[sq::kStBadBounds]) return SQ_ERR_CUDA;
  *lo = b[0];
  *hi = b[1];
  return SQ_OK;
}

int sq_node_bounds(sq_handle* h, double* lo_out, double* hi_out) {
  if (!h || !lo_out || !hi_out) return SQ_ERR_INVALID_ARG;
  if (h->bounds_mode != SQ_BOUNDS_PER_NODE) return sq::fail(h, SQ_ERR_INVALID_ARG, "not in per-node bounds mode");
  if (!h->bounds_ready) return sq::fail(h, SQ_ERR_STATE, "no per-node bounds yet");
  std::vector<double> b(2 * size_t(h->Nd));
  SQ_CUDA_TRY(h, cudaMemcpyAsync(b.data(), h->d.nbnd, sizeof(double) * b.size(), cudaMemcpyDeviceToHost, h->stream));
  SQ_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  for (int q = 0; q < h->Nd; ++q) {
    lo_out[q] = b[2 * q];
    hi_out[q] = b[2 * q + 1];
  }
  return SQ_OK;
}

int sq_moments_copy(sq_handle* h, double* host_out) {
  if (!h || !host_out) return SQ_ERR_INVALID_ARG;
  if (!h->moments_ready) return sq::fail(h, SQ_ERR_STATE, "no moments yet");
  size_t bytes = sizeof(double) * size_t(h->Nd) * size_t(h->geo.n_pl + 1) * SQ_N_MOMENTS;
  SQ_CUDA_TRY(h, cudaMemcpyAsync(host_out, h->d.mom, bytes, cudaMemcpyDeviceToHost, h->stream));
  SQ_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return SQ_OK;
}

long long sq_kernel_launches(const sq_handle* h) { return h ? h->launches : 0; }

int sq_tune_step(sq_handle* h, int n_warps, int wave_tiles, int reps, double* ms_per_tile) {
  if (!h || n_warps < 0 || n_warps > 8 || wave_tiles < 0 || reps < 0) return SQ_ERR_INVALID_ARG;
  h->step_warps = n_warps;
  // new wave split over the handle's tiles, within the buffers sized at setup, evenly spread
  const int ntl = h->tile_end - h->tile_begin;
  const int cap = (wave_tiles > 0) ? std::min(wave_tiles, h->wave_cap) : h->wave_cap;
  const int nwaves = std::max(1, (ntl + cap - 1) / std::max(1, cap));
  const int per = std::max(1, (ntl + nwaves - 1) / nwaves);
  h->waves.clear();
  for (int t0 = h->tile_begin; t0 < h->tile_end; t0 += per) h->waves.push_back({t0, std::min(per, h->tile_end - t0), nullptr});
  h->wave_rows.clear();
  int rc = sq::measure_wave_rows(h);
  if (rc != SQ_OK) return rc;
  if (reps > 0 && ms_per_tile) {
    // the timed launches reuse the sweep buffers of wave 0; the moments table is not touched
    if (!h->bounds_ready) return sq::fail(h, SQ_ERR_STATE, "sq_tune_step timing needs the bounds (sq_moments first)");
    double ms = 0.0;
    rc = sq::time_step_launch(h, reps, &ms);
    if (rc != SQ_OK) return rc;
    *ms_per_tile = h->waves.empty() ? 0.0 : ms / h->waves[0].ntiles;
  }
  return SQ_OK;
}

int sq_keep_lists(sq_handle* h, int enable) {
  if (!h) return SQ_ERR_INVALID_ARG;
  h->keep_lists = enable != 0;
  return SQ_OK;
}

int sq_step_launch_counts(const sq_handle* h, long long* counts) {
  if (!h || !counts) return SQ_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i) counts[i] = h->step_variant[i];
  return SQ_OK;
}

int sq_kernel_timing(sq_handle* h, int enable) {
  if (!h) return SQ_ERR_INVALID_ARG;
  h->timing = enable != 0;
  if (h->timing)
    for (int k = 0; k < 3; ++k) h->t_launches[k] = 0, h->t_ms[k] = 0, h->t_bytes[k] = 0;
  return SQ_OK;
}

int sq_kernel_timing_read(const sq_handle* h, int kid, long long* launches, double* total_ms, double* algo_bytes) {
  if (!h || kid < 0 || kid > 2) return SQ_ERR_INVALID_ARG;
  if (launches) *launches = h->t_launches[kid];
  if (total_ms) *total_ms = h->t_ms[kid];
  if (algo_bytes) *algo_bytes = h->t_bytes[kid];
  return SQ_OK;
}

void sq_destroy(sq_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

const char* sq_last_error(const sq_handle* h) {
  if (h) return h->err.empty() ? "no error" : h->err.c_str();
  return g_setup_err.c_str();
}

}  // extern "C"
