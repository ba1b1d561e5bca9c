// Internal declarations of the GB300 SQ library (not part of the C ABI).
//
// Device layout (node-batched lattice tiles)
//   * The N_d grid nodes are grouped into tiles of b x b x b adjacent nodes (B = b^3).
//   * A tile's union window U is the box of absolute (unwrapped) lattice points
//     [o - m, o + b - 1 + m] per axis (o = tile origin); every node window W_q of the tile
//     is a sub-box of U. A Chebyshev column t_q^j of every node of the tile is stored on U,
//     node index innermost: T[pt][node], pt = (uz * Uy + uy) * Ux + ux. Entries outside the
//     node's own window are held at exactly zero, which realises the restriction H_q of
//     Sec. 4 (zero extension) while the B nodes share each stencil load of V_eff and of the
//     projector tables.
//   * Atoms: each atom's projector channels are sampled once on the atom's support box in
//     absolute lattice coordinates; a periodic image is the same table shifted by s * n.
//   * Per tile, the atom images whose support box meets U are listed (TileEntry), and per
//     4x4x4 brick of U the entries meeting the brick (used by the per-point nonlocal apply).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sq_api.h"

namespace sq {

constexpr int kMaxNo = 6;        // largest FD half-order supported
constexpr int kBrick = 4;        // brick side in points
constexpr int kMaxCh = 8;        // projector channels per atom
constexpr int kThreads = 256;    // block size of the tile kernels
constexpr int kMaxU = 2 * 64 + 8; // largest union-window extent (m <= 64, b = 2, x padded to 4)
constexpr size_t kLzDotCap = 8192;   // doubles of the Lanczos dot-product chunk partials

struct AtomTab {
  int lo[3];        // support box corner (absolute lattice coordinates of the base image)
  int dim[3];       // support box extent
  int nch;          // channels
  int nchp;         // channels padded to a multiple of 4 (table stride per point)
  int ch0;          // first channel in the per-channel arrays
  int pad;
  long long off;    // table offset; channel c of box point li at off + li * nchp + c
  double R[3];      // base image position (wrapped into the cell)
  float dlo[3];     // lo_a h_a - R_a: x_a - R_a of box point l is l_a h_a + dlo[a] (any image)
  int pad2;
};

struct TileEntry {
  int atom;         // atom index
  int s[3];         // image shift in cells
  int row0;         // first projector row of this entry in the tile's P / A arrays
  int pad;
};

// An atom image as seen from one 4^3 brick (2 x int4, read warp-uniformly in the sweep):
//   r0 = {off, row0, ch0, nch | nchp << 8}   off = table index of the brick corner
//   r1 = {dx, dy, mask_lo, mask_hi}          box extents; 64-bit mask of the brick points
//                                            (bit a + 4 b + 16 c) inside the support sphere
// Point (a, b, c) of the brick has its channel group at off + ((c * dy + b) * dx + a) * nchp.

// Everything a tile kernel needs, passed by value.
struct Geo {
  int n[3];
  int m[3];
  int b, B;
  int U[3];
  int Upts;
  int nbr[3];       // bricks per axis
  int nbricks;
  int tiles[3];
  int n_tiles;
  int n_o;
  int n_atoms;
  double h[3];
  double L[3];
  double dV;
  double lap0;                    // -1/2 sum_a w0 / h_a^2
  double lap[3][kMaxNo + 1];      // -1/2 w_p / h_a^2
  double grd[3][kMaxNo + 1];      // g_p / h_a
  float lap0f;                    // float copies used by the FP32 sweep (constant-bank operands)
  float lapf[3][kMaxNo + 1];
  float grdf[3][kMaxNo + 1];
  int e_cap;                      // entries per tile (capacity)
  int r_cap;                      // projector rows per tile (capacity)
  int br_cap;                     // entries per brick (capacity)
  int n_pl;
  int nslab;                      // slabs per tile: y-rows of bricks (kBrick y-planes, all x, all z)
};

struct Wave {
  int tile0;           // first global tile of this wave (when ids is null)
  int ntiles;          // tiles in this wave
  const int* ids;      // device list of global tile indices, or null for tile0 + i
};

// Per-wave device buffers (sized for the largest wave).
struct WaveBufs {
  TileEntry* entries = nullptr;   // [wt][e_cap]
  int* n_entries = nullptr;       // [wt]
  int* n_rows = nullptr;          // [wt]
  int* brick_list = nullptr;      // [wt][nbricks][br_cap]
  int* brick_n = nullptr;         // [wt][nbricks]
  int4* brick_rec = nullptr;      // [wt][nbricks][br_cap][2] per-brick image records
  float4* brick_d0 = nullptr;     // [wt][nbricks][br_cap] x - R of the record's brick corner (FP32 W table)
  int4* brick_tma = nullptr;      // [wt][nbricks][br_cap] (atom, box-local x, y, z of the brick corner)
  int* slab_n = nullptr;          // [wt][nslab] projector rows meeting each slab (y-row of bricks)
  int* slab_map = nullptr;        // [wt][nslab][r_cap] slab row -> tile row
  void* T[3] = {nullptr, nullptr, nullptr};   // Real [wt][Upts][B]
  void* W = nullptr;              // Real [wt][3][Upts][B]
  void* A = nullptr;              // Real [wt][r_cap][B]  chi_row(x_q)
  void* P = nullptr;              // Real [wt][r_cap][B]  gamma |dOmega| chi^T t (Lanczos apply)
  void* Pg[2] = {nullptr, nullptr};   // double [wt][r_cap][B]  gamma |dOmega| chi^T t^j, ping-pong
  double* Spart = nullptr;        // [wt][nslab][B][9]
};

struct Dev {
  double* v64 = nullptr;          // V_eff (N_d)
  float* v32 = nullptr;
  AtomTab* atoms = nullptr;       // [n_atoms]
  double* gdv = nullptr;          // per channel: [gamma*dV, l, m, width, rcut, 0]
  double* gdv64 = nullptr;        // gamma * dV per channel
  double* rcmax = nullptr;        // per atom: largest projector radius
  float* gdv32 = nullptr;
  double* chi64 = nullptr;        // projector tables
  float* chi32 = nullptr;
  float* chi32s = nullptr;        // mixed: each FP32 table value as a TF32 (hi, lo) pair
  double* mom = nullptr;          // [N_d][n_pl+1][17]
  double* R = nullptr;            // [n_pl+1] node sums of rho^j
  double* cosF = nullptr;         // [M] sum'_j cos(j theta_k) R^j
  double* coef = nullptr;         // [3][n_pl+1] c, d, s at the last contraction mu
  double* scal = nullptr;         // scalars: mu, bounds, partial sums ...
  double* part = nullptr;         // contraction partials
  double* rho = nullptr;          // [N_d]
  int* status = nullptr;          // device status words
  double* lzV = nullptr;          // Lanczos basis [(k+1)][nst][Upts][B]
  double* lzW = nullptr;          // Lanczos work vector [nst][Upts][B]
  double* lzP = nullptr;          // projections of the Lanczos vector [nst][r_cap][B]
  double* lzC = nullptr;          // Gram-Schmidt coefficients / alpha, beta [cols][...]
  int* lz_tiles = nullptr;        // sample tile ids [nst]
  double* lzdot = nullptr;        // chunk partials of the Lanczos dot products of small waves [kLzDotCap]
  // per-node bounds mode (SQ_BOUNDS_PER_NODE)
  double* nbnd = nullptr;         // [N_d][2] effective (lo, hi) of every node
  double* ncoef = nullptr;        // [N_d][2] step coefficients (ca = 2 / zeta_q, cd = ca lap0 - 2 chi_q / zeta_q)
  double* nF = nullptr;           // [N_d][M] sum'_j cos(j theta_k) rho_q^j
  double* nrow = nullptr;         // [N_d][20] contraction terms per node
  double* costab = nullptr;       // [4 M] cos(pi t / (2 M))
  double* npart = nullptr;        // [1024] partial electron counts
  void* nV = nullptr;             // Lanczos wave buffers of the per-node bounds
  void* nW = nullptr;
  void* nP = nullptr;
  double* nC = nullptr;
};

}  // namespace sq

struct sq_handle {
  sq_instance_desc desc;          // copy (host pointers cleared after setup)
  sq::Geo geo;
  int precision = SQ_FP64;
  int bounds_mode = SQ_BOUNDS_LANCZOS;
  int M = 2048;
  int lanczos_k = 40;
  double kT = 0, n_e = 0;
  double lam_lo = 0, lam_hi = 0;   // effective bounds (those the recurrence realises)
  double lap_offset = 0;            // constant-mode eigenvalue of the stored stencil weights
  double hscal[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  bool bounds_ready = false;
  bool moments_ready = false;
  int Nd = 0;
  double vol = 0;
  cudaStream_t stream = nullptr;
  std::vector<sq::AtomTab> atoms_h;
  std::vector<double> rcmax_h;      // per atom: support radius (its table slot is sized for it)
  int lz_cap = 0;                   // Lanczos sample-tile capacity of the buffers
  int nlz_wave = 0;                 // tiles per Lanczos wave of the per-node bounds
  long long table_len = 0;
  int n_ch_total = 0;
  bool proj4 = false;               // every atom has at most 4 projector channels (one group per image)
  std::vector<sq::Wave> waves;
  std::vector<int> wave_rows;       // per wave: most projector rows of a slab (shared-memory size)
  std::vector<int> wave_recs;       // per wave: most atom images meeting one brick (staged step)
  int tile_begin = 0, tile_end = 0;   // tiles this handle sweeps (node partition)
  int wave_cap = 0;
  sq::Dev d;
  sq::WaveBufs wb;
  sq::WaveBufs lzb;                 // list buffers of the Lanczos sample tiles (default bounds)
  // what wb's lists (and W, A) describe: the wave, the atom positions (epoch, bumped by
  // sq_update_atoms) and whether W was built too; a sweep of the same wave reuses them
  struct ListsKey {
    int tile0 = -1, ntiles = 0;
    const int* ids = nullptr;
    long long epoch = -1;
    bool full = false;
  } lists_key;
  long long atoms_epoch = 0;
  bool keep_lists = false;          // sq_keep_lists: reuse the lists of unchanged atoms
  long long lz_lists_epoch = -1;    // atom epoch of the Lanczos sample tiles' lists in lzb
  std::vector<int> lanczos_tiles;
  long long launches = 0;
  // step-kernel launches by variant: [0] projections staged in shared memory, tensor-core
  // projector phases; [1] shared memory, scalar phases; [2] projections in global memory;
  // [3] the TMA-staged step (sq_step_tma.cu)
  long long step_variant[4] = {0, 0, 0, 0};
  // tensor maps of the TMA-staged step: t buffers (x, y, z sticks, brick), W, projector tables
  CUtensorMap tmT[3][4];
  CUtensorMap tmW;
  CUtensorMap tmChi;
  bool tma_ok = false;              // the maps exist and the instance fits the staged step
  bool step_staged = false;         // SQ_STEP_KERNEL=staged: the TMA-staged step where it applies
  int stage_recs_cap = 16;          // SQ_STAGE_RECS: atom images per stage of the staged step
  bool stage_wait_test = false;     // SQ_STAGE_WAIT_TEST=1: the staged step's copy wait runs out (tests)
  int step_rows_cap = 0;            // most projector rows a step block stages in shared memory
  int step_warps = 0;               // warps per step block (0: the brick-count rule; set by the tuner)
  // optional event timing of the sweep kernels
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, double>> ev_pending;   // (kernel class, algorithmic bytes) per pair
  long long t_launches[3] = {0, 0, 0};
  double t_ms[3] = {0, 0, 0};
  double t_bytes[3] = {0, 0, 0};
  size_t bytes = 0;
  std::vector<void*> allocs;
  std::string err;
};

namespace sq {

// Named host-side range around a phase of the pipeline (setup, bounds, each sweep wave, Fermi
// search, contraction, batch, request), shown on a profiler's timeline; header-only NVTX v3,
// which costs nothing when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Spectral scaling of the recurrence from bounds [lo, hi] (sq_api.cu): writes the step
// coefficients and the effective bounds used by the Fermi search and the contraction.
int set_bounds(sq_handle* h, double lo, double hi);
// The same scaling on the device from the Lanczos interval in scal[8], scal[9] (sq_lanczos.cu)
int set_bounds_device(sq_handle* h);
// per-wave slab row counts and brick image counts (sq_sweep.cu): size the step kernels' shared
// memory, once per layout
int measure_wave_rows(sq_handle* h);
// the TMA-staged FP32 step (sq_step_tma.cu): tensor maps (after the buffers exist), its shared
// memory for a slab row count and a brick image count, and one launch on t buffers ic, ip
constexpr size_t kStepTmaSmemMax = 220 * 1024;
int make_step_maps(sq_handle* h);
size_t step_tma_smem_bytes(int rows, int cap_rec);
int launch_step_tma(sq_handle* h, const Wave& w, dim3 grid, int ic, int ip, float* Tn, const double* Pg, double* Pgn,
                    int mode, int rows, int cap_rec);
// one recurrence step launch (mode 1) of wave 0 with the handle's current settings, timed with
// CUDA events on its stream (sq_sweep.cu; the autotuner's measurement)
int time_step_launch(sq_handle* h, int reps, double* ms_out);

// error helpers
int fail(sq_handle* h, int code, const std::string& msg);
#define SQ_CUDA_TRY(h, call)                                                              \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return ::sq::fail((h), SQ_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)
#define SQ_LAUNCH_CHECK(h)                                                                \
  do {                                                                                    \
    (h)->launches++;                                                                      \
    cudaError_t e_ = cudaGetLastError();                                                  \
    if (e_ != cudaSuccess)                                                                \
      return ::sq::fail((h), SQ_ERR_CUDA, std::string("kernel launch (") + __FILE__ + ":" + std::to_string(__LINE__) + "): " + cudaGetErrorString(e_)); \
  } while (0)

int dev_alloc(sq_handle* h, void** p, size_t bytes);
// event timing helpers (sq_api.cu): open a pair before a launch, collect after a sync
cudaEvent_t timing_begin(sq_handle* h, int kid, double bytes);
void timing_end(sq_handle* h, cudaEvent_t start);
int timing_collect(sq_handle* h);

// setup kernels (sq_setup.cu)
int build_tables(sq_handle* h);
int init_node_tables(sq_handle* h);   // per-node bounds mode: cosine table, neutral node bounds
// the lists, A, W and t^0 of a wave in wb; with reuse, the lists and W of the same wave and atom
// positions built by the previous sweep are kept (only A, the projection buffers and t^0 are
// rewritten)
int build_wave_lists(sq_handle* h, const Wave& w, bool reuse);

// sweep (sq_sweep.cu)
int run_sweep(sq_handle* h);
int step_rows_smem_max(int precision);
// out = H_q v for every node column of the wave's tiles (FP64), P = projection scratch
// H_q v on the sample tiles of the Lanczos bounds (FP64 or FP32 vectors, matching tables)
int launch_apply_h(sq_handle* h, const Wave& w, const double* v, double* out, double* P, const WaveBufs& b);
int launch_apply_h(sq_handle* h, const Wave& w, const float* v, float* out, float* P, const WaveBufs& b);
// entries / brick lists of a wave only (no A, W, t^0), into b (the sweep's wb by default)
int build_wave_entries(sq_handle* h, const Wave& w, WaveBufs* b = nullptr);

// bounds / Fermi level / contraction (sq_reduce.cu)
int run_lanczos(sq_handle* h);
// k-step Lanczos of every node column of a wave (start 0: hash vector, 1: e_q); see sq_lanczos.cu
template <typename Real>
int lanczos_columns(sq_handle* h, const Wave& w, int start, int k, Real* V, Real* W, Real* P, double* C,
                    WaveBufs* b);
int run_fermi(sq_handle* h, double* mu_out);
// per-node bounds mode (sq_lanczos.cu, sq_reduce.cu)
int run_lanczos_nodes(sq_handle* h);
int run_fermi_nodes(sq_handle* h, double* mu_out);
int run_contraction_nodes(sq_handle* h, double mu, double* rho_dev, double* sums_host);
int run_node_sums(sq_handle* h, double* R_out);
int run_fermi_sums(sq_handle* h, const double* R_host, double* mu_out);
int run_contraction(sq_handle* h, double mu, double* rho_dev, double* sums_host);
// Fermi level + contraction with mu and the outputs kept on the device (sq_reduce.cu)
int run_fermi_contraction_device(sq_handle* h);

// status word indices
enum StatusWord { kStOverflow = 0, kStNoBracket = 1, kStTimeout = 2, kStNoConverge = 3, kStBadBounds = 4, kStCount = 5 };

}  // namespace sq
