// The Chebyshev step of Sec. 4 in FP32 with its inputs staged in shared memory by the tensor
// memory accelerator (TMA), one 4^3 brick at a time:
//     t^{j+1} = 2 Hhat_q t^j - t^{j-1},   Hhat_q = (H_q - chi I) / zeta,
//     H_q t = -1/2 sum_a (D2_a / h_a^2) t + V_eff t + sum_rows gamma |dOmega| chi (chi^T t),
// with the nonlocal-stress partial sum_u W_b (grad_a t^j)(u) of S^j_ab.
//
// One block of 8 warps per (slab = y-row of bricks, tile) walks the slab's bricks in order. Per
// brick one elected lane issues cp.async.bulk.tensor loads (completion counted on one mbarrier)
// of
//   - three "sticks" of t^j: the brick with its 6-point halo along x, along y and along z
//     (16 x 4 x 4 points each; points outside the union window come back as zeros, which is the
//     zero extension of the restriction H_q, so no stencil tap needs a bounds check and every
//     tap is a shared-memory load at a constant offset),
//   - the three W_b fields and t^{j-1} on the brick,
//   - for every atom image that meets the brick, its projector values (TF32 hi/lo pairs of the
//     four channels) on the brick's 64 points, straight from the atom's table (table slots have
//     one box shape per instance, so one tensor map covers all atoms; box points outside the
//     table come back as zeros). A stage holds cap_rec images; a brick that meets more (dense
//     cells, small periodic cells) takes them in chunks, each one more phase of the mbarrier,
//     for the apply and again (last chunk first) for the projections.
// Then
//   A  the nonlocal apply Y = X Pg^j on TF32 tensor cores (3-term hi/lo split, FP32
//      accumulation): M = 64 brick points, N = 8 nodes, K = 4 channels per image; the 8 warps
//      take (m-tile = z-plane, half of the images) and the two halves are summed in phase B,
//   B  stencil, V_eff, apply, window mask, recurrence update and the S partials: one 8-byte
//      (node pair) shared load per tap, 8 warps x 32 lanes x 2 nodes = the brick's 512 columns,
//   C  the projections gamma |dOmega| X^T t^{j+1} of the new column on tensor cores (M = 4
//      images x 4 channels, N = 8 nodes, K = 64 points split over two warps). Each K half keeps
//      its own FP32 slab sums, and every (row, node) of a half belongs to one lane, so the sums are
//      plain adds in a fixed order (no atomics, the same bits on every run); once per slab both
//      halves go into the tile's FP64 projection sums.
// Waits on the mbarrier are bounded (about a second of clock cycles); a wait that runs out sets
// the timeout status word, and the block waits (again bounded) for its copies before leaving.
#include <cuda.h>

#include "sq_device.cuh"

namespace sq {

namespace {

constexpr int kTmaWarps = 8;
constexpr int kTmaThreads = 32 * kTmaWarps;
constexpr int kStickFloats = 16 * 4 * 4 * 8;   // a brick and its halo along one axis, 8 nodes
constexpr int kCoreFloats = 4 * 4 * 4 * 8;     // one brick, 8 nodes
constexpr int kRecFloats = 64 * 8;             // one image's 4 channels (hi, lo) at 64 points
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// orders this thread's earlier generic-proxy shared accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// spin on the phase with the given parity for at most kWaitCycles clock cycles
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

// 5-D tiled TMA load of one box into shared memory, completion counted on bar
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1, int c2,
                                            int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }

}  // namespace

// Shared-memory bytes of one k_step_tma block: staged records (cap_rec images), sticks, W,
// t^{j-1}, the apply halves, t^{j+1}, the slab's projections (staged, and the two accumulated
// halves), the brick's record headers, the S reduction and the mbarrier.
size_t step_tma_smem_bytes(int rows, int cap_rec) {
  return size_t(cap_rec) * kRecFloats * 4 + 3 * kStickFloats * 4 + 3 * kCoreFloats * 4 + kCoreFloats * 4 +
         2 * kCoreFloats * 4 + kCoreFloats * 4 + size_t(rows) * 8 * 4 * 3 + size_t(cap_rec) * 16 +
         kTmaWarps * 8 * 9 * 4 + 16;
}

template <int NO>
__global__ void __launch_bounds__(kTmaThreads, 2)
k_step_tma(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap my,
           const __grid_constant__ CUtensorMap mz, const __grid_constant__ CUtensorMap mp,
           const __grid_constant__ CUtensorMap mw, const __grid_constant__ CUtensorMap mchi, Geo g, Wave w,
           float* __restrict__ Tn, const double* __restrict__ Pg, double* __restrict__ Pg_next,
           const float* __restrict__ gdv, const int4* __restrict__ brec, const int4* __restrict__ btma,
           const int* __restrict__ slab_n, const int* __restrict__ slab_map, const int* __restrict__ bn,
           const float* __restrict__ v, const double* __restrict__ scal, int mode, double* __restrict__ Spart,
           int rows_smem, int cap_rec, const double* __restrict__ ncoef, int* __restrict__ status,
           int extra_tx) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int wrx[kMaxU], wry[kBrick], wrz[kMaxU];
  float* s_chi = reinterpret_cast<float*>(smem_raw);                 // [cap_rec][64 points][8]
  float* s_xs = s_chi + size_t(cap_rec) * kRecFloats;                // [4 z][4 y][16 x][8]
  float* s_ys = s_xs + kStickFloats;                                 // [4 z][16 y][4 x][8]
  float* s_zs = s_ys + kStickFloats;                                 // [16 z][4 y][4 x][8]
  float* s_w = s_zs + kStickFloats;                                  // [3][64][8]
  float* s_tp = s_w + 3 * kCoreFloats;                               // [64][8]
  float* s_y = s_tp + kCoreFloats;                                   // [2][64][8] apply halves
  float* s_tn = s_y + 2 * kCoreFloats;                               // [64][8] t^{j+1}
  float* s_pst = s_tn + kCoreFloats;                                 // [rows][8] Pg^j (slab rows)
  float* s_ps = s_pst + size_t(rows_smem) * 8;                       // [2][rows][8] projections of t^{j+1}
  int4* s_rec = reinterpret_cast<int4*>(s_ps + size_t(rows_smem) * 16);  // [cap_rec] record headers
  float* s_red = reinterpret_cast<float*>(s_rec + cap_rec);          // [8 warps][8 nodes][9]
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_red + kTmaWarps * 8 * 9);

  const int slab = blockIdx.x, tl = blockIdx.y, t = wave_tile(w, tl);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nsr = slab_n[(size_t)tl * g.nslab + slab];
  // a copy wait of this sweep already ran out: its results are void, skip the work
  if (*reinterpret_cast<volatile int*>(status + kStTimeout)) return;
  if (nsr > rows_smem) {   // a launch sized for another layout (e.g. a stale graph): refuse
    if (threadIdx.x == 0) atomicOr(status + kStOverflow, 4);
    return;
  }
  const int* smap = slab_map + ((size_t)tl * g.nslab + slab) * g.r_cap;
  double* Pn = Pg_next + (size_t)tl * g.r_cap * 8;
  const double* Pt = Pg + (size_t)tl * g.r_cap * 8;
  int o[3];
  tile_origin(g, t, o);
  const double f = (mode == 0) ? 0.5 : 1.0;
  const float ca = float(f * scal[4]), cd = float(f * scal[6]), cc = (mode == 1) ? 1.f : 0.f;
  const int Uy = g.U[1], Uz = g.U[2];
  const size_t tbase = (size_t)tl * g.Upts * 8;
  const bool project = (mode != 2);
  const uint32_t bar = smem_addr(s_bar);

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
  for (int i = threadIdx.x; i < nsr * 8; i += blockDim.x) {
    s_pst[i] = float(Pt[smap[i >> 3] * 8 + (i & 7)]);
    s_ps[i] = 0.f;
    s_ps[size_t(rows_smem) * 8 + i] = 0.f;
  }
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();

  // phase B roles: lane = (node pair np2: nodes 2 np2, 2 np2 + 1 at x offsets 0, 1; x point xa2;
  // y parity yb2), warp = brick iteration: points (xa2, 2 (warp % 2) + yb2, warp / 2)
  const int np2 = lane & 3, xa2 = (lane >> 2) & 3, yb2 = lane >> 4;
  const int pb = 2 * (warp & 1) + yb2, pc = warp >> 1;
  const int qo2[3] = {0, np2 & 1, np2 >> 1};
  bool valid2[2];
  {
    const int qa[3] = {0, qo2[1], qo2[2]}, qb[3] = {1, qo2[1], qo2[2]};
    valid2[0] = node_valid(g, o, qa);
    valid2[1] = node_valid(g, o, qb);
  }
  // step coefficients of the lane's two nodes: the block's (shared bounds) or each node's own
  float caA = ca, cdA = cd, caB = ca, cdB = cd;
  if (ncoef) {
    auto own = [&](int qx, float& c_a, float& c_d) {
      const int qq[3] = {qx, qo2[1], qo2[2]};
      if (!node_valid(g, o, qq)) return;
      const int node = (o[0] + qx) + g.n[0] * ((o[1] + qo2[1]) + g.n[1] * (o[2] + qo2[2]));
      c_a = float(f * ncoef[2 * node]);
      c_d = float(f * ncoef[2 * node + 1]);
    };
    own(0, caA, cdA);
    own(1, caB, cdB);
  }
  const int pidx = (xa2 + 4 * pb + 16 * pc) * 8 + 2 * np2;   // the lane's (point, node pair) in a brick array
  const float* xsp = s_xs + ((pc * 4 + pb) * 16 + xa2 + 6) * 8 + 2 * np2;
  const float* ysp = s_ys + ((pc * 16 + pb + 6) * 4 + xa2) * 8 + 2 * np2;
  const float* zsp = s_zs + (((pc + 6) * 4 + pb) * 4 + xa2) * 8 + 2 * np2;
  // MMA fragment roles (m16n8k8): g8 = lane / 4, t4 = lane % 4
  const int g8 = lane >> 2, t4 = lane & 3;

  float sb[18];   // S partials of nodes 2 np2, 2 np2 + 1 over the lane's points of all bricks
#pragma unroll
  for (int k = 0; k < 18; ++k) sb[k] = 0.f;

  const int nbx = g.nbr[0], nbz = g.nbr[2], nbs = nbx * nbz;
  auto brick_index = [&](int bi) -> size_t {
    return (size_t)tl * g.nbricks + (size_t)((bi / nbx) * g.nbr[1] + slab) * nbx + bi % nbx;
  };
  // the next brick's image count (every thread) and, in warp 0, the TMA boxes of its first 64
  // images (lane, lane + 32): loaded one brick ahead, so issuing a brick's copies waits on no
  // global load
  int nb_next = bn[brick_index(0)];
  int4 tr_a = make_int4(0, 0, 0, 0), tr_b = make_int4(0, 0, 0, 0);   // this brick's
  int4 nx_a = tr_a, nx_b = tr_b;                                       // the next brick's
  if (warp == 0 && project) {
    const int n0 = min(nb_next, 64);
    if (lane < n0) nx_a = btma[brick_index(0) * g.br_cap + lane];
    if (lane + 32 < n0) nx_b = btma[brick_index(0) * g.br_cap + lane + 32];
  }
  uint32_t parity = 0;
  // one stage load: warp 0 arms the mbarrier with the byte count and issues the copies of images
  // [k0, k0 + nc) of brick bidx (and with core, the sticks, W and t^{j-1}); every thread copies
  // the images' record headers
  auto issue = [&](size_t bidx, int x0, int y0, int z0, int k0, int nc, bool core) {
    if (warp == 0) {
      if (lane == 0) {
        // extra_tx > 0 (a test of the bounded wait) arms the phase for bytes that never arrive
        const uint32_t bytes = uint32_t((core ? 3 * kStickFloats * 4 + 3 * kCoreFloats * 4 : 0) +
                                        (core && mode == 1 ? kCoreFloats * 4 : 0) + nc * kRecFloats * 4 + extra_tx);
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, bytes);
      }
      __syncwarp();
      if (core && lane == 0) {
        tma_load_5d(smem_addr(s_xs), &mx, bar, 0, x0 - 6, y0, z0, tl);
        tma_load_5d(smem_addr(s_ys), &my, bar, 0, x0, y0 - 6, z0, tl);
        tma_load_5d(smem_addr(s_zs), &mz, bar, 0, x0, y0, z0 - 6, tl);
        tma_load_5d(smem_addr(s_w), &mw, bar, 0, x0, y0, z0, 3 * tl);
        if (mode == 1) tma_load_5d(smem_addr(s_tp), &mp, bar, 0, x0, y0, z0, tl);
      }
      for (int k = lane; k < nc; k += 32) {
        // (atom, box-local corner x, y, z) of image k0 + k: prefetched for images lane, lane + 32
        const int kk = k0 + k;
        const int4 tr = (kk == lane) ? tr_a : (kk == lane + 32) ? tr_b : btma[bidx * g.br_cap + kk];
        tma_load_5d(smem_addr(s_chi + size_t(k) * kRecFloats), &mchi, bar, 0, tr.y, tr.z, tr.w, tr.x);
      }
    }
    for (int k = threadIdx.x; k < nc; k += blockDim.x) s_rec[k] = brec[(bidx * g.br_cap + k0 + k) * 2];
  };
  // wait for the armed phase; false (the whole block) when the bounded wait ran out somewhere
  auto wait_stage = [&]() -> bool {
    const bool ok = mbar_wait_bounded(bar, parity);
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) atomicOr(status + kStTimeout, 1);
      mbar_wait_bounded(bar, parity);   // let copies still in flight land before the block exits
      return false;
    }
    parity ^= 1u;
    return true;
  };

  for (int bi = 0; bi < nbs; ++bi) {
    const int bx = bi % nbx, bz = bi / nbx, by = slab;
    const size_t bidx = brick_index(bi);
    const int nb = project ? nb_next : 0;   // images of the brick (the moments-only step needs none)
    // images beyond the stage's capacity come in further chunks of cap_rec (dense cells)
    const int nchunk = (nb + cap_rec - 1) / cap_rec;
    const int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrick;
    tr_a = nx_a;
    tr_b = nx_b;
    issue(bidx, x0, y0, z0, 0, min(nb, cap_rec), true);
    if (bi + 1 < nbs) nb_next = bn[brick_index(bi + 1)];
    // inputs of phase B that do not come through the stage
    const int ux = x0 + xa2, uy = y0 + pb, uz = z0 + pc;
    const bool inU = (uy < Uy) && (uz < Uz);
    const float vloc = inU ? v[wrz[uz] + wry[pb] + wrx[ux]] : 0.f;
    if (!wait_stage()) return;

    if (project) {
      // phase A: Y[64 points][8 nodes] = X[64][4 nb] Pg^j[4 nb][8]; m-tile = z-plane mt, K step =
      // 2 images x 4 channels (K = t4 -> image k2 + t4 / 2, channel 2 (t4 % 2); K = t4 + 4 -> the
      // next channel); rows g8 and g8 + 8 = brick points 16 mt + g8 and 16 mt + g8 + 8
      const int mt = warp & 3, kh = warp >> 2, ch = 2 * (t4 & 1);
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      for (int c = 0; c < nchunk; ++c) {
        const int nc = min(cap_rec, nb - c * cap_rec);
        if (c > 0) {
          __syncthreads();   // chunk c - 1 is read
          issue(bidx, x0, y0, z0, c * cap_rec, nc, false);
          if (!wait_stage()) return;
        }
        for (int k2 = 2 * kh; k2 < nc; k2 += 4) {
          const int kr = k2 + (t4 >> 1);
          uint4 xa = make_uint4(0u, 0u, 0u, 0u), xc = make_uint4(0u, 0u, 0u, 0u);
          uint32_t bh[2] = {0u, 0u}, bl[2] = {0u, 0u};
          if (kr < nc) {
            const int4 r0 = s_rec[kr];
            const int nch = r0.w & 0xff, prow = int(unsigned(r0.w) >> 16);
            const float p0 = (ch < nch) ? s_pst[(prow + ch) * 8 + g8] : 0.f;
            const float p1 = (ch + 1 < nch) ? s_pst[(prow + ch + 1) * 8 + g8] : 0.f;
            split_tf32(p0, bh[0], bl[0]);
            split_tf32(p1, bh[1], bl[1]);
            const float* xb = s_chi + size_t(kr) * kRecFloats + (16 * mt + g8) * 8 + 2 * ch;
            xa = *reinterpret_cast<const uint4*>(xb);
            xc = *reinterpret_cast<const uint4*>(xb + 64);
          }
          const uint32_t ah[4] = {xa.x, xc.x, xa.z, xc.z}, al[4] = {xa.y, xc.y, xa.w, xc.w};
          mma_tf32(acc, al, bh);   // small terms first
          mma_tf32(acc, ah, bl);
          mma_tf32(acc, ah, bh);
        }
      }
      float* yk = s_y + kh * kCoreFloats;
      *reinterpret_cast<float2*>(yk + (16 * mt + g8) * 8 + 2 * t4) = make_float2(acc[0], acc[1]);
      *reinterpret_cast<float2*>(yk + (16 * mt + g8 + 8) * 8 + 2 * t4) = make_float2(acc[2], acc[3]);
      if (warp == 0 && bi + 1 < nbs) {   // the next brick's TMA boxes (see above)
        const int n1 = min(nb_next, 64);
        const size_t b1 = brick_index(bi + 1) * g.br_cap;
        if (lane < n1) nx_a = btma[b1 + lane];
        if (lane + 32 < n1) nx_b = btma[b1 + lane + 32];
      }
    }
    __syncthreads();

    // phase B
    {
      const size_t e = ((size_t)(uz * Uy + uy) * g.U[0] + ux) * 8 + 2 * np2;
      const bool inyz = inU && (unsigned)(uy - qo2[1]) <= (unsigned)(2 * g.m[1]) &&
                        (unsigned)(uz - qo2[2]) <= (unsigned)(2 * g.m[2]);
      const bool in0 = inyz && valid2[0] && (unsigned)ux <= (unsigned)(2 * g.m[0]);
      const bool in1 = inyz && valid2[1] && (unsigned)(ux - 1) <= (unsigned)(2 * g.m[0]);
      float2 tn = make_float2(0.f, 0.f);
      if (in0 || in1) {
        const float2 tc = lds2(xsp);
        const float2 w0 = lds2(s_w + pidx), w1 = lds2(s_w + kCoreFloats + pidx), w2 = lds2(s_w + 2 * kCoreFloats + pidx);
        float2 y = make_float2(0.f, 0.f);   // off-diagonal part of H t^j
        float2 gr[3];
        const float* sp[3] = {xsp, ysp, zsp};
        constexpr int kStep[3] = {8, 32, 128};   // floats between neighbouring points along x, y, z
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          gr[a] = make_float2(0.f, 0.f);
#pragma unroll
          for (int pp = 1; pp <= NO; ++pp) {
            const float2 fp = lds2(sp[a] + pp * kStep[a]);
            const float2 fm = lds2(sp[a] - pp * kStep[a]);
            const float wl = g.lapf[a][pp], wg = g.grdf[a][pp];
            y.x += wl * (fp.x + fm.x);
            y.y += wl * (fp.y + fm.y);
            gr[a].x += wg * (fp.x - fm.x);
            gr[a].y += wg * (fp.y - fm.y);
          }
        }
        if (project) {
          const float2 ya = lds2(s_y + pidx), yb = lds2(s_y + kCoreFloats + pidx);
          y.x += ya.x + yb.x;
          y.y += ya.y + yb.y;
          const float2 tp = (mode == 1) ? lds2(s_tp + pidx) : make_float2(0.f, 0.f);
          const float dgA = cdA + caA * vloc, dgB = cdB + caB * vloc;
          if (in0) tn.x = caA * y.x + dgA * tc.x - cc * tp.x;
          if (in1) tn.y = caB * y.y + dgB * tc.y - cc * tp.y;
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
      }
      if (project) {
        if (inU) *reinterpret_cast<float2*>(Tn + tbase + e) = tn;
        *reinterpret_cast<float2*>(s_tn + pidx) = tn;
      }
    }
    __syncthreads();

    if (project) {
      // phase C: Pg^{j+1}[4 nb rows][8] += X^T[4 nb][64 points] t^{j+1}[64][8]; m-tile = 4 images
      // (row g8 -> image m4 + g8 / 2, channel 2 (g8 % 2); row g8 + 8 -> the next channel), K step =
      // points 8 ks + t4 and 8 ks + t4 + 4, the two warps of an m-tile split the 8 K steps. The
      // chunks run last to first: the last one is still staged from phase A.
      const int kh = warp >> 2, ch = 2 * (g8 & 1);
      float* psk = s_ps + size_t(kh) * rows_smem * 8;
      for (int c = nchunk - 1; c >= 0; --c) {
        const int nc = min(cap_rec, nb - c * cap_rec);
        if (c < nchunk - 1) {
          issue(bidx, x0, y0, z0, c * cap_rec, nc, false);   // chunk c + 1 was read (sync below)
          if (!wait_stage()) return;
        }
        for (int m4 = 4 * (warp & 3); m4 < nc; m4 += 16) {
          const int kr = m4 + (g8 >> 1);
          const bool rv = kr < nc;
          const float* xb = s_chi + size_t(rv ? kr : 0) * kRecFloats + t4 * 8 + 2 * ch;
          float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int ks = 4 * kh + s;
            uint4 xa = make_uint4(0u, 0u, 0u, 0u), xc = make_uint4(0u, 0u, 0u, 0u);
            if (rv) {
              xa = *reinterpret_cast<const uint4*>(xb + 64 * ks);
              xc = *reinterpret_cast<const uint4*>(xb + 64 * ks + 32);
            }
            const uint32_t ah[4] = {xa.x, xa.z, xc.x, xc.z}, al[4] = {xa.y, xa.w, xc.y, xc.w};
            uint32_t bh[2], bl[2];
            split_tf32(s_tn[(8 * ks + t4) * 8 + g8], bh[0], bl[0]);
            split_tf32(s_tn[(8 * ks + t4 + 4) * 8 + g8], bh[1], bl[1]);
            mma_tf32(d, al, bh);
            mma_tf32(d, ah, bl);
            mma_tf32(d, ah, bh);
          }
          if (rv) {
            const int4 r0 = s_rec[kr];
            const int nch = r0.w & 0xff, prow = int(unsigned(r0.w) >> 16);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int cch = ch + (i >> 1);
              if (cch < nch) psk[(prow + cch) * 8 + 2 * t4 + (i & 1)] += d[i] * gdv[r0.z + cch];
            }
          }
        }
        __syncthreads();   // chunk c is read (and after the last, the stage is free for the next brick)
      }
    } else {
      __syncthreads();
    }
  }

  // S partials: the 8 point lanes of each node pair (xor 4, 8, 16), then the warps, in FP64
#pragma unroll
  for (int k = 0; k < 18; ++k) {
    float sv = sb[k];
    sv += __shfl_xor_sync(0xffffffffu, sv, 4);
    sv += __shfl_xor_sync(0xffffffffu, sv, 8);
    sv += __shfl_xor_sync(0xffffffffu, sv, 16);
    if (lane < 4) s_red[(warp * 8 + 2 * lane + k / 9) * 9 + k % 9] = sv;
  }
  __syncthreads();
  for (int k2 = threadIdx.x; k2 < 8 * 9; k2 += blockDim.x) {
    const int qq = k2 / 9, k = k2 % 9;
    double sv = 0.0;
    for (int wv = 0; wv < kTmaWarps; ++wv) sv += double(s_red[(wv * 8 + qq) * 9 + k]);
    Spart[(((size_t)tl * g.nslab + slab) * 8 + qq) * 9 + k] = sv;
  }
  if (project) {
    for (int i = threadIdx.x; i < nsr * 8; i += blockDim.x) {
      const double s = double(s_ps[i]) + double(s_ps[size_t(rows_smem) * 8 + i]);
      if (s != 0.0) atomicAdd(&Pn[smap[i >> 3] * 8 + (i & 7)], s);
    }
  }
}

// ------------------------------------------------------------------------------ host side
namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 5-D FP32 tensor {8, X, Y, Z, N} (innermost first) with 32-byte points, and a box of it
bool encode5(EncodeTiled fn, CUtensorMap* m, void* base, const unsigned long long dims[5],
             const unsigned box[5]) {
  cuuint64_t gd[5], gs[4];
  cuuint32_t bd[5], es[5];
  for (int i = 0; i < 5; ++i) {
    gd[i] = dims[i];
    bd[i] = box[i];
    es[i] = 1;
  }
  gs[0] = dims[0] * 4;
  for (int i = 1; i < 4; ++i) gs[i] = gs[i - 1] * dims[i];
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, base, gd, gs, bd, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace

// Tensor maps of the staged step (SQ_MIXED): the three t buffers (x, y, z sticks and the brick),
// the W fields and the TF32 (hi, lo) projector tables. The staged step applies when every atom
// has at most 4 channels (8 floats per table point) and all table slots have one box shape and
// follow each other in atom order; otherwise (or when the driver offers no encoder) h->tma_ok
// stays false and the step kernel of sq_sweep.cu runs.
int make_step_maps(sq_handle* h) {
  h->tma_ok = false;
  if (h->precision != SQ_MIXED || !h->proj4 || h->geo.b != 2) return SQ_OK;
  const Geo& g = h->geo;
  unsigned long long slot[3] = {0, 0, 0};
  for (size_t J = 0; J < h->atoms_h.size(); ++J) {
    const AtomTab& at = h->atoms_h[J];
    if (J == 0)
      for (int a = 0; a < 3; ++a) slot[a] = (unsigned long long)at.dim[a];
    const unsigned long long pts = slot[0] * slot[1] * slot[2];
    if (at.nch <= 0 || at.nchp != 4 || (unsigned long long)at.off != J * pts * 4) return SQ_OK;
    for (int a = 0; a < 3; ++a)
      if ((unsigned long long)at.dim[a] != slot[a]) return SQ_OK;
  }
  EncodeTiled fn = encode_fn();
  if (!fn) return SQ_OK;
  const unsigned long long wt = (unsigned long long)h->wave_cap;
  const unsigned long long tdims[5] = {8, (unsigned long long)g.U[0], (unsigned long long)g.U[1],
                                       (unsigned long long)g.U[2], wt};
  const unsigned bx[5] = {8, 16, 4, 4, 1}, by[5] = {8, 4, 16, 4, 1}, bz[5] = {8, 4, 4, 16, 1}, bc[5] = {8, 4, 4, 4, 1};
  for (int i = 0; i < 3; ++i) {
    if (!encode5(fn, &h->tmT[i][0], h->wb.T[i], tdims, bx) || !encode5(fn, &h->tmT[i][1], h->wb.T[i], tdims, by) ||
        !encode5(fn, &h->tmT[i][2], h->wb.T[i], tdims, bz) || !encode5(fn, &h->tmT[i][3], h->wb.T[i], tdims, bc))
      return SQ_OK;
  }
  const unsigned long long wdims[5] = {8, (unsigned long long)g.U[0], (unsigned long long)g.U[1],
                                       (unsigned long long)g.U[2], 3 * wt};
  const unsigned bw[5] = {8, 4, 4, 4, 3};
  if (!encode5(fn, &h->tmW, h->wb.W, wdims, bw)) return SQ_OK;
  if (!h->atoms_h.empty()) {
    const unsigned long long cdims[5] = {8, slot[0], slot[1], slot[2], (unsigned long long)h->atoms_h.size()};
    if (!encode5(fn, &h->tmChi, h->d.chi32s, cdims, bc)) return SQ_OK;
  } else {
    h->tmChi = h->tmW;   // never read: no atom, no record
  }
  h->tma_ok = true;
  return SQ_OK;
}

template <int NO>
static void launch_tma(sq_handle* h, const Wave& w, dim3 grid, size_t smem, int ic, int ip, float* Tn, const double* Pg,
                       double* Pgn, int mode, int rows, int cap_rec) {
  const double* ncoef = (h->bounds_mode == SQ_BOUNDS_PER_NODE) ? h->d.ncoef : nullptr;
  k_step_tma<NO><<<grid, kTmaThreads, smem, h->stream>>>(
      h->tmT[ic][0], h->tmT[ic][1], h->tmT[ic][2], h->tmT[ip][3], h->tmW, h->tmChi, h->geo, w, Tn, Pg, Pgn,
      h->d.gdv32, h->wb.brick_rec, h->wb.brick_tma, h->wb.slab_n, h->wb.slab_map, h->wb.brick_n, h->d.v32,
      h->d.scal, mode, h->wb.Spart, rows, cap_rec, ncoef, h->d.status, h->stage_wait_test ? 16 : 0);
}

// Launches the staged step on buffers T[ic] (t^j), T[ip] (t^{j-1}) -> Tn; rows / cap_rec size the
// shared memory (the wave's largest slab row count and brick image count).
int launch_step_tma(sq_handle* h, const Wave& w, dim3 grid, int ic, int ip, float* Tn, const double* Pg, double* Pgn,
                    int mode, int rows, int cap_rec) {
  const size_t smem = step_tma_smem_bytes(rows, cap_rec);
  h->step_variant[3]++;
  auto set_attr = [&](const void* fn) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kStepTmaSmemMax));
  };
  cudaError_t e = cudaSuccess;
  switch (h->geo.n_o) {
    case 1: e = set_attr((const void*)k_step_tma<1>); if (e == cudaSuccess) launch_tma<1>(h, w, grid, smem, ic, ip, Tn, Pg, Pgn, mode, rows, cap_rec); break;
    case 2: e = set_attr((const void*)k_step_tma<2>); if (e == cudaSuccess) launch_tma<2>(h, w, grid, smem, ic, ip, Tn, Pg, Pgn, mode, rows, cap_rec); break;
    case 3: e = set_attr((const void*)k_step_tma<3>); if (e == cudaSuccess) launch_tma<3>(h, w, grid, smem, ic, ip, Tn, Pg, Pgn, mode, rows, cap_rec); break;
    case 4: e = set_attr((const void*)k_step_tma<4>); if (e == cudaSuccess) launch_tma<4>(h, w, grid, smem, ic, ip, Tn, Pg, Pgn, mode, rows, cap_rec); break;
    case 5: e = set_attr((const void*)k_step_tma<5>); if (e == cudaSuccess) launch_tma<5>(h, w, grid, smem, ic, ip, Tn, Pg, Pgn, mode, rows, cap_rec); break;
    default: e = set_attr((const void*)k_step_tma<6>); if (e == cudaSuccess) launch_tma<6>(h, w, grid, smem, ic, ip, Tn, Pg, Pgn, mode, rows, cap_rec); break;
  }
  if (e != cudaSuccess) return fail(h, SQ_ERR_CUDA, std::string("k_step_tma attribute: ") + cudaGetErrorString(e));
  SQ_LAUNCH_CHECK(h);
  return SQ_OK;
}

}  // namespace sq
