/*
 * sq_api.h -- C ABI of the GB300 infinite-cell Clenshaw-Curtis Spectral Quadrature (SQ)
 * library: electron density, band / entropy / nonlocal energies and the density-matrix
 * (kinetic + nonlocal) Hellmann-Feynman stress of an orthorhombic periodic cell, following
 * Sharma, Hamel, Bethkenhagen, Pask, Suryanarayana, "Real-space formulation of the stress
 * tensor for O(N) density functional theory" (arXiv 2006.03697), Sec. 4 and App. A; also the
 * Gauss SQ density and the Green-Kubo viscosity the paper uses in Sec. 5.
 *
 * Problem statement (Sec. 4). The cell is discretised by a uniform grid K_Omega of N_d nodes,
 * node i at (ix h0, iy h1, iz h2), h_a = L_a / n_a. For every node q the nodal Hamiltonian
 * H_q is the restriction of the infinite-crystal grid Hamiltonian
 *     H = -1/2 Lap_h + V_eff + sum_{I in R^3} sum_lm gamma_Jl |dOmega| chi_Ilm chi_Ilm^T
 * to the node's region of influence, the cube of half-width R_cut around q
 * (m_a = floor(R_cut / h_a + 1e-9) points per side, zero extension outside it).
 * With Hhat_q = (H_q - chi I) / zeta and the Chebyshev columns
 *     t^0 = e_q,  t^1 = Hhat_q e_q,  t^{j+1} = 2 Hhat_q t^j - t^{j-1}   (j < n_pl),
 * the library forms per node and per j = 0..n_pl the moments
 *     rho^j = e_q^T t^j,  K^j_ab = e_q^T grad_a,q grad_b,q t^j,  N^j = e_q^T V_nl,q t^j,
 *     S^j_ab = sum_I e_q^T V^I_nl,q (X_b,q - R_Ib) grad_a,q t^j,
 * finds the Fermi level mu from N_e = 2 sum_q sum'_j c^j(mu) rho_q^j, and contracts
 *     rho_q  = (2/|dOmega|) sum'_j c^j rho_q^j
 *     E_band = 2 sum_q sum'_j (chi c^j + zeta d^j) rho_q^j          (App. A)
 *     E_s    = 2 kT sum_q sum'_j s^j rho_q^j      (-TS; s = g ln g + (1-g) ln(1-g))
 *     E_nl   = 2 sum_q sum'_j c^j N_q^j
 *     sigma  = [2 sum sum' c^j K^j - 2 sum sum' c^j (delta N^j + 2 S^j)] / |Omega|
 * where c^j, d^j, s^j are the Chebyshev coefficients of the Fermi-Dirac function g, of r g(r)
 * and of the entropy function in the scaled variable, and the primed sum halves j = 0.
 *
 * Conventions
 *   - Units: Hartree atomic units (Ha, bohr); spin-unpolarised (factor 2).
 *   - Arrays are row-major; grid arrays are x fastest: i = ix + n0 (iy + n1 iz).
 *   - sigma is returned row-major 3x3 in Ha/bohr^3 (sigma[3*a + b]).
 *   - Every call returns an int status (SQ_OK = 0). The library never aborts or traps; on
 *     error sq_last_error() describes the failure. No kernel of the library waits on another
 *     kernel or on the host. The one device wait is the TMA-staged step's wait for its own
 *     copies into shared memory (SQ_MIXED with SQ_STEP_KERNEL=staged): it gives up after about
 *     2e9 clock cycles (about a second), and the sweep then returns SQ_ERR_TIMEOUT (sq_moments,
 *     sq_batch_run). The environment variable SQ_STAGE_WAIT_TEST=1, read by sq_setup, makes that
 *     wait run out on purpose (for tests; the copies still complete).
 *   - The caller owns every host buffer passed in or out; the library copies inputs during
 *     sq_setup and owns all device memory of a handle until sq_destroy.
 *   - A handle is used by one host thread at a time. Work is issued on desc->stream
 *     (a cudaStream_t; NULL selects the legacy default stream).
 */
#ifndef SQ_API_H
#define SQ_API_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SQ_OK 0
#define SQ_ERR_INVALID_ARG 1   /* a descriptor field or pointer is out of range       */
#define SQ_ERR_OOM 2           /* device or host allocation failed                    */
#define SQ_ERR_CUDA 3          /* a CUDA runtime call failed                           */
#define SQ_ERR_NO_BRACKET 4    /* N(mu) - N_e has no sign change on the bisection bracket */
#define SQ_ERR_TIMEOUT 5       /* a bounded device wait (staged step copies) ran out    */
#define SQ_ERR_STATE 6         /* call out of order (e.g. contraction before moments)  */

/* precision modes */
#define SQ_FP64 0    /* FP64 recurrence, projectors and moments                          */
#define SQ_MIXED 1   /* FP32 recurrence and moment products, projector products on TF32
                        tensor cores with a hi/lo split (about 2^-21 relative), FP32
                        Lanczos vectors for the bounds; FP64 node and cross-thread sums,
                        Gram-Schmidt coefficients, Fermi search and contraction          */

/* spectral bound modes (the paper takes chi, zeta from the extreme eigenvalues of H_q) */
#define SQ_BOUNDS_LANCZOS 0   /* k-step Lanczos on sample regions, widened (default)   */
#define SQ_BOUNDS_GIVEN 1     /* lambda_lo / lambda_hi taken from the descriptor        */
#define SQ_BOUNDS_PER_NODE 2  /* Sec. 4 literally: chi_q, zeta_q from the extreme eigenvalues
                                 of each node's own H_q (k-step Lanczos on every node, widened
                                 as the shared interval); the Fermi search and the contraction
                                 use each node's own coefficients c_q^j(mu), d_q^j, s_q^j.
                                 Not combined with a node partition.                      */

/* Moments per node and Chebyshev index (sq_moments_copy layout) */
#define SQ_N_MOMENTS 17  /* rho, K_xx K_yy K_zz K_yz K_xz K_xy, N, S_ab (8 + 3a + b) */

/* Gaussian Kleinman-Bylander projector of one species (stand-in for the pseudopotential
 * projectors chi_Jlm of Eqs. sigmaIII / E_nl):
 *   l = 0: chi = (pi w^2)^(-3/4) exp(-r^2 / (2 w^2))
 *   l = 1: chi_m = sqrt(2)/w * d_m * (pi w^2)^(-3/4) exp(-r^2 / (2 w^2)),  m = x, y, z
 * zero for r > rcut (rcut <= 0 selects 7 w). */
typedef struct {
  int l;          /* 0 or 1                                     */
  double width;   /* w > 0 (bohr)                               */
  double gamma;   /* gamma_Jl (Ha)                              */
  double rcut;    /* support radius (bohr)                      */
} sq_proj;

typedef struct {
  double L[3];                 /* orthorhombic cell sides (bohr), > 0                          */
  int n[3];                    /* nodes per side, >= 1                                          */
  int n_o;                     /* FD half-order 1..6 (2 n_o-order central stencils)            */
  const double* v_eff;         /* host, N_d values (x fastest), finite                          */
  int n_atoms;                 /* >= 0                                                          */
  const double* pos;           /* host, [n_atoms][3] bohr, any real values (periodic)           */
  const int* species;          /* host, [n_atoms] in [0, n_species)                             */
  int n_species;               /* >= 1 when n_atoms > 0                                         */
  const int* proj_offset;      /* host, [n_species + 1]: projectors of species s are
                                  proj[proj_offset[s] .. proj_offset[s+1])                      */
  const sq_proj* proj;         /* host, [proj_offset[n_species]]                                */
  double kT;                   /* smearing sigma = kT > 0 (Ha)                                  */
  double n_e;                  /* electrons per cell, 0 < n_e < 2 N_d                           */
  double r_cut;                /* truncation radius (bohr); m_a >= 1 required                   */
  int n_pl;                    /* Chebyshev degree >= 1 (terms j = 0..n_pl)                     */
  int precision;               /* SQ_FP64 | SQ_MIXED                                            */
  int bounds_mode;             /* SQ_BOUNDS_LANCZOS | SQ_BOUNDS_GIVEN                           */
  double lambda_lo, lambda_hi; /* used with SQ_BOUNDS_GIVEN; lambda_lo < lambda_hi               */
  int cheb_quad_M;             /* Chebyshev-Gauss points for c, d, s (<= 0 selects 2048)        */
  int lanczos_k;               /* Lanczos steps (<= 0 selects 40)                               */
  void* stream;                /* cudaStream_t or NULL                                          */
  int part_rank, part_count;   /* node partition (Sec. 4: the nodes of K_Omega are divided among
                                  processors and every SQ sum is a sum over them): with
                                  part_count > 0 the handle sweeps only tile range part_rank of
                                  part_count equal contiguous ranges of the 2 x 2 x 2-node tiles
                                  (tile t = tx + T0 (ty + T1 tz)); 0 = the whole cell. See
                                  sq_node_sums / sq_fermi_level_sums for the exchange step.      */
} sq_instance_desc;

typedef struct {
  double E_band;   /* 2 sum_q sum' (chi c + zeta d) rho^j  (Ha)      */
  double E_s;      /* -TS (Ha)                                       */
  double E_nl;     /* nonlocal energy (Ha)                           */
  double F;        /* E_band + E_s (Mermin free energy of these terms) */
  double N_check;  /* |dOmega| sum_q rho_q (should equal n_e)        */
  double mu;       /* Fermi level used (Ha)                          */
} sq_energies;

typedef struct sq_handle sq_handle;

/* Validates desc, copies every input to the device, samples the projectors on their support
 * boxes, builds the per-tile atom-image lists and allocates the recurrence buffers.
 * On success *out owns all device memory of the instance. Errors: SQ_ERR_INVALID_ARG,
 * SQ_ERR_OOM, SQ_ERR_CUDA (then *out is NULL). */
int sq_setup(const sq_instance_desc* desc, sq_handle** out);

/* Spectral bounds (SQ_BOUNDS_LANCZOS: device Lanczos, Sec. 4 chi_q / zeta_q), then the
 * Chebyshev sweep over every node (Sec. 4 three-term recurrence) and the moment table.
 * Asynchronous on the handle's stream. Errors: SQ_ERR_CUDA, SQ_ERR_OOM. */
int sq_moments(sq_handle* h);

/* Fermi level by FP64 bisection on N(mu) = 2 sum'_j c^j(mu) R^j, R^j = sum_q rho_q^j, on
 * [lambda_lo - 40 kT, lambda_hi + 40 kT] until the bracket is < 1e-13 max(1, |mu|) or 200
 * steps; runs on the device and synchronises the stream. Errors: SQ_ERR_STATE (no moments),
 * SQ_ERR_NO_BRACKET, SQ_ERR_CUDA. */
int sq_fermi_level(sq_handle* h, double* mu_out);

/* Resident state for a trajectory (successive quantum-MD snapshots of one cell): gives the
 * handle new atom positions pos [n_atoms][3] and a new V_eff [N_d] (host, copied before
 * return) for the same cell, grid, species and projectors. The device buffers, stream and
 * projector-table slots of the handle are kept (each atom's table slot is sized at sq_setup
 * for any position); the base images, support boxes and projector tables are rebuilt, and
 * with SQ_BOUNDS_LANCZOS the bounds are recomputed by the next sq_moments (sample tiles from
 * the new V_eff). Results equal those of a fresh sq_setup of the new snapshot. The moments
 * must be recomputed (sq_moments) before the Fermi level or a contraction. Synchronises.
 * Errors: SQ_ERR_INVALID_ARG (NULL or non-finite input), SQ_ERR_CUDA. */
int sq_update_atoms(sq_handle* h, const double* pos, const double* v_eff);

/* Fixed atoms across calls (e.g. SCF iterations of Sec. 5, where only V_eff changes): with
 * enable != 0, the sweep keeps the per-tile atom-image lists, the brick records and the W_b
 * table it built for the current atom positions across sq_moments calls (so do the Lanczos
 * bounds for the lists of their sample tiles), instead of rebuilding them in every call. They
 * depend on the positions only: sq_update_atoms with moved atoms discards them, with the same
 * positions and a new V_eff it keeps them. Kept only when the handle's tiles form one wave
 * (sq_footprint_bytes up to about 64 GiB of per-tile buffers). Off by default, where every
 * sq_moments rebuilds them as a new snapshot needs. Results are identical either way.
 * Errors: SQ_ERR_INVALID_ARG. */
int sq_keep_lists(sq_handle* h, int enable);

/* Node partition (part_count > 0): the moments of the nodes outside the handle's tile range
 * are zero, so R^j and every contraction output are this part's share of the node sums of
 * Sec. 4, and the parts add up to the whole cell. The Fermi level needs the whole-cell sums:
 *   sq_node_sums        R_out [n_pl + 1] (host) = sum over this part's nodes of rho_q^j
 *                       (fixed order); synchronises. Errors: SQ_ERR_STATE (no moments).
 *   sq_fermi_level_sums the bisection of sq_fermi_level on the caller's R_host [n_pl + 1]
 *                       (the sum of every part's sq_node_sums, e.g. one allreduce of n_pl + 1
 *                       doubles); synchronises. Errors: SQ_ERR_STATE, SQ_ERR_INVALID_ARG
 *                       (NULL or non-finite R_host), SQ_ERR_NO_BRACKET.
 * Each part then calls sq_density_energy_stress / sq_pressure at that mu and the parts' E_band,
 * E_s, E_nl, N_check, E_pot, sigma and pressure add up (one allreduce of 15 doubles); rho_out
 * holds this part's nodes (zero elsewhere). Unpartitioned handles may use both calls too. */
int sq_node_sums(sq_handle* h, double* R_out);
int sq_fermi_level_sums(sq_handle* h, const double* R_host, double* mu_out);

/* Contraction at mu (Sec. 4 rho_q and stress sums, App. A band energy). Host outputs:
 * rho_out [N_d] or NULL, e_out or NULL, sigma_out [9] or NULL. Synchronises the stream. */
int sq_density_energy_stress(sq_handle* h, double mu, double* rho_out, sq_energies* e_out,
                             double* sigma_out);

/* Same with DEVICE outputs (e.g. torch data_ptr): rho_dev [N_d] doubles or NULL, sigma_dev [9]
 * doubles or NULL; energies (if e_out) are still written to host memory. Does not synchronise
 * unless e_out is non-NULL. */
int sq_density_energy_stress_dev(sq_handle* h, double mu, double* rho_dev, sq_energies* e_out,
                                 double* sigma_dev);

/* Pressure only (App. A, Eq. ON:Pressure and its SQ form) restricted to the kinetic and
 * nonlocal terms: the band term -4 sum_q sum'_j (chi c^j + zeta d^j) rho^j_q = -2 E_band less its
 * V_eff part, and the nonlocal term -2 sum_q w_q^T V_nl,q (sum' c^j t^j + 2 (X - R).grad sum' c^j t^j):
 *   P = (2 (E_band - E_pot) + E_nl + 4 sum_q sum'_j c^j (S^j_xx + S^j_yy + S^j_zz)_q) / (3 |Omega|)
 * in Ha/bohr^3, with E_pot = |dOmega| sum_q V_eff(x_q) rho_q (Ha), the V_eff part of the band
 * energy, which the paper's formula pairs with the exchange-correlation and electrostatic
 * terms outside this library. Needs no second derivatives of the density matrix (the K^j
 * moments are not used); equals -tr(sigma)/3 when sigma's kinetic moments are taken with
 * the second-difference operator of H, up to the Chebyshev truncation of E_band.
 * Host outputs: pressure_out (required), e_pot_out or NULL. Synchronises the stream.
 * Errors: SQ_ERR_STATE (no moments), SQ_ERR_INVALID_ARG (NULL pressure_out, non-finite mu). */
int sq_pressure(sq_handle* h, double mu, double* pressure_out, double* e_pot_out);

/* Bounds in use (after sq_moments in Lanczos mode); in SQ_BOUNDS_PER_NODE mode the smallest
 * lower and the largest upper node bound. */
int sq_get_bounds(const sq_handle* h, double* lambda_lo, double* lambda_hi);

/* SQ_BOUNDS_PER_NODE: every node's effective interval [lo_q, hi_q] (host, [N_d] each, x fastest)
 * after sq_moments: the one the recurrence realises (chi_q -+ zeta_q after the FP32-exact
 * scaling of SQ_MIXED and the stencil's constant-mode offset), which the Fermi search and the
 * contraction use. Errors: SQ_ERR_INVALID_ARG (NULL, other bounds modes), SQ_ERR_STATE. */
int sq_node_bounds(sq_handle* h, double* lo_out, double* hi_out);

/* Copies the moment table [N_d][n_pl + 1][SQ_N_MOMENTS] (FP64, host) for inspection. */
int sq_moments_copy(sq_handle* h, double* host_out);

/* Device bytes sq_setup would allocate for desc (0 if desc is invalid); used for admission. */
size_t sq_footprint_bytes(const sq_instance_desc* desc);

/* Number of CUDA kernels the handle launched since sq_setup (all calls). */
long long sq_kernel_launches(const sq_handle* h);

/* Launches of the Chebyshev step kernel since sq_setup, by variant, into counts[4] (host):
 *   counts[0]  projections of the block's atom images staged in shared memory, projector
 *              phases on tensor cores (SQ_MIXED, at most 4 channels per atom)
 *   counts[1]  staged in shared memory, scalar projector phases (SQ_FP64, or > 4 channels)
 *   counts[2]  projections read and accumulated in global memory (a block meets more
 *              projector rows than shared memory holds: dense atoms, large R_cut)
 *   counts[3]  the TMA-staged step (SQ_MIXED, at most 4 channels per atom, one projector
 *              radius per instance, selected by SQ_STEP_KERNEL=staged): every input of a brick
 *              (t^j with its stencil halo, W, t^{j-1}, the projector values of the images meeting
 *              it) copied into shared memory by the tensor memory accelerator
 * The environment variables, read by sq_setup: SQ_STEP_SMEM_ROWS lowers the row count above
 * which a block uses global memory (tuning and tests); SQ_STEP_KERNEL=staged puts a mixed handle
 * on the TMA-staged step where its shared memory fits, SQ_STAGE_RECS (1..64, default 16) sets
 * the atom images per stage. Errors: SQ_ERR_INVALID_ARG. */
int sq_step_launch_counts(const sq_handle* h, long long* counts);

/* Autotuning hook of the step kernel: n_warps warps per step block (1..8; 0 = the default,
 * the count that leaves the fewest idle warps over a slab's bricks) and at most wave_tiles tiles
 * per launch (0 = as many as the buffers sized at sq_setup hold; waves are spread evenly over the
 * handle's tiles). The settings stay with the handle. With reps > 0 and ms_per_tile non-NULL,
 * also times reps recurrence-step launches of the first wave with CUDA events on the handle's
 * stream and returns milliseconds per tile and step; with more than one wave this includes the
 * rebuild of the wave's lists and W table that every sweep then pays, spread over its n_pl + 1
 * steps (one wave keeps them across evaluations) (needs the bounds: after sq_moments, or
 * SQ_BOUNDS_GIVEN; the sweep buffers are reused, the moments table is not touched).
 * Synchronises. Errors: SQ_ERR_INVALID_ARG, SQ_ERR_STATE, SQ_ERR_CUDA. */
int sq_tune_step(sq_handle* h, int n_warps, int wave_tiles, int reps, double* ms_per_tile);

/* Kernel classes of the Chebyshev sweep timed by sq_kernel_timing (see below). */
#define SQ_K_STENCIL 0   /* H t^j, window mask, recurrence update, S partials          */
#define SQ_K_PROJECT 1   /* chi^T t^{j+1} per atom image                                */
#define SQ_K_MOMENTS 2   /* rho^j, K^j, N^j, S^j per node                               */

/* enable != 0: record a CUDA event pair on the handle's stream around every launch of the
 * sweep kernels of later sq_moments calls and reset the accumulators; enable == 0: stop. */
int sq_kernel_timing(sq_handle* h, int enable);

/* For kernel class kid: launches timed, their summed event time (ms), and the algorithmic
 * bytes they moved (stencil only: 4 B per float / 8 B per double for each read of t^j and
 * t^{j-1} and each write of t^{j+1}, per node and region point; 0 for other classes). */
int sq_kernel_timing_read(const sq_handle* h, int kid, long long* launches, double* total_ms,
                          double* algo_bytes);

/* Fermi level without any device allocation. The paper has no counterpart: this is a
 * service for callers that cannot call cudaMalloc (an allocator that is locked or at its
 * budget, a plug-in that must leave the process's device heap alone). It runs the same
 * bisection as sq_fermi_level on a moment table the caller owns:
 *   mom_dev      device, [n_nodes][n_pl + 1][SQ_N_MOMENTS] FP64 (the sq_moments_copy layout;
 *                only slot 0, rho^j, is read)
 *   lambda_lo/hi the spectral bounds the table was computed with (sq_get_bounds)
 *   kT, n_e      smearing and electron count; cheb_quad_M <= 0 selects 2048
 *   stream       cudaStream_t or NULL; the call is asynchronous on it
 *   mu_dev       device, 1 double: receives mu, or NaN when N(mu) - N_e has no sign change
 * Its scratch (node sums and cosine sums) lives in one fixed file-scope device array of
 * (SQ_NOALLOC_MAX_NPL + 1 + SQ_NOALLOC_MAX_M + 32) doubles (about 73 KB) that every GPU
 * loading the library holds until exit; n_pl > SQ_NOALLOC_MAX_NPL or M > SQ_NOALLOC_MAX_M is
 * rejected with SQ_ERR_INVALID_ARG. No cudaMalloc / cudaFree or allocating library call is
 * made. Every call made outside stream capture looks up the array's device address with the
 * calling device current (so the address stays right after a device reset reloads the module);
 * a call inside a capture reuses the address of the last uncaptured call on that device, so make
 * the first call on each device (and the first after a reset) outside any stream capture: a
 * first call inside one returns SQ_ERR_STATE. Every call rewrites the whole scratch; calls that
 * overlap on the GPU share it and race. */
#define SQ_NOALLOC_MAX_NPL 1024
#define SQ_NOALLOC_MAX_M 8192
int sq_fermi_level_noalloc(const double* mom_dev, int n_nodes, int n_pl, double lambda_lo, double lambda_hi,
                           double kT, double n_e, int cheb_quad_M, void* stream, double* mu_dev);

/* Batched evaluation of independent instances (uneven snapshots): every handle runs its whole
 * pipeline (sq_moments, sq_fermi_level, contraction at that mu) on its own host thread, at most
 * max_concurrent (<= 0: n) at a time, so their kernels overlap on the device. Give each handle
 * its own stream (desc->stream) or they serialise. Outputs (host, may be NULL): mu_out [n],
 * e_out [n], sigma_out [n][9]. Each result is identical to evaluating that handle alone.
 * Returns the first non-zero status (details in that handle's sq_last_error). */
int sq_batch_evaluate(sq_handle* const* hs, int n, int max_concurrent, double* mu_out, sq_energies* e_out,
                      double* sigma_out);

/* One CUDA graph for a batch of handles (uneven instances: atom counts, cells, R_cut, n_pl,
 * precisions may differ; SQ_BOUNDS_LANCZOS or SQ_BOUNDS_GIVEN): sq_batch_create captures each
 * member's whole evaluation (Lanczos bounds, sweep with moments, Fermi level, contraction) as
 * one branch of the graph, with nothing crossing to the host inside it; sq_batch_run launches
 * the graph once, waits, and writes the members' results (host, may be NULL): mu_out [n],
 * e_out [n], sigma_out [n][9]; the members' moments and density (sq_moments_copy,
 * sq_density_energy_stress at another mu) are then available as after sq_moments. Members need
 * their own non-NULL streams and must not be used elsewhere while the batch runs. After
 * sq_update_atoms on members, sq_batch_run evaluates the new snapshots (re-capturing the graph
 * when a member's wave layout grew). Errors: SQ_ERR_INVALID_ARG (NULL, repeated handles or
 * streams, per-node bounds), SQ_ERR_CUDA, SQ_ERR_NO_BRACKET (first failing member; its handle's
 * sq_last_error, sq_batch_last_error says which). */
typedef struct sq_batch sq_batch;
int sq_batch_create(sq_handle* const* hs, int n, sq_batch** out);
/* The graph's schedule: members i, i + C, i + 2C, ... run one after another as chain i, the C
 * chains side by side (C = chains; 0 or >= n: every member in its own branch, the default; 1:
 * all members in turn). Captures the graph again. Results do not depend on it. Errors:
 * SQ_ERR_INVALID_ARG, SQ_ERR_CUDA. */
int sq_batch_set_chains(sq_batch* b, int chains);
int sq_batch_run(sq_batch* b, double* mu_out, sq_energies* e_out, double* sigma_out);
const char* sq_batch_last_error(const sq_batch* b);
void sq_batch_destroy(sq_batch* b);

/* Request loop with continuous batching (one GPU). Requests are admitted in submission order
 * as soon as their device footprint (sq_footprint_bytes) fits under hbm_budget_bytes next to
 * those in flight and fewer than max_inflight run; each admitted request runs setup, moments,
 * Fermi level and contraction on its own stream and host thread and is destroyed afterwards
 * (see sq_server_submit_traj for requests that keep their state on the device).
 * A request larger than the whole budget completes with status SQ_ERR_OOM. */
typedef struct sq_server sq_server;
typedef struct {
  long long tag;         /* the caller's tag from sq_server_submit           */
  int status;            /* SQ_OK or the failing call's status               */
  double mu;             /* Fermi level (Ha)                                  */
  sq_energies energies;  /* as sq_density_energy_stress                       */
  double sigma[9];       /* Ha/bohr^3, row-major                             */
  double latency_ms;     /* submit -> result available                       */
  char error[128];       /* sq_last_error text when status != SQ_OK          */
} sq_result;
int sq_server_create(size_t hbm_budget_bytes, int max_inflight, sq_server** out);
/* Copies every input of desc (desc->stream is ignored); returns SQ_ERR_INVALID_ARG if desc
 * does not validate, SQ_ERR_STATE after sq_server_destroy has begun. Non-blocking. */
int sq_server_submit(sq_server* s, const sq_instance_desc* desc, long long tag);
/* Moves up to max_results finished results to out (host), waiting up to timeout_ms for the
 * first one; *n_out receives the count. */
int sq_server_poll(sq_server* s, sq_result* out, int max_results, int timeout_ms, int* n_out);
/* A request that belongs to trajectory traj (>= 0): successive snapshots of one cell (same
 * grid, species, projectors, kT, n_e, r_cut, n_pl, precision and bounds mode; new positions
 * and V_eff). The trajectory's first request sets up a handle that stays resident on the device;
 * its later requests move that handle's atoms in place (sq_update_atoms) instead of setting up
 * and destroying one, and run one at a time in submission order (requests of other
 * trajectories may go ahead of a request whose trajectory is busy). A request whose other
 * fields differ from the resident handle's replaces it. Idle resident handles count against
 * hbm_budget_bytes and are released, least recently used first, when a request needs the
 * memory, and all of them by sq_server_destroy. Errors: as sq_server_submit; traj < 0 is
 * SQ_ERR_INVALID_ARG. */
int sq_server_submit_traj(sq_server* s, const sq_instance_desc* desc, long long tag, long long traj);
/* Requests queued or running (-1 for NULL). */
int sq_server_pending(sq_server* s);
/* Trajectory handles resident on the device (-1 for NULL). */
int sq_server_resident(sq_server* s);
/* Stops admitting, finishes every queued and running request, frees the server (results not
 * polled are dropped). */
void sq_server_destroy(sq_server* s);

/* Gauss Spectral Quadrature of the electron density (the SQ variant the paper uses for the SCF
 * density, Sec. 5; cited there without formulas). For every node q: k-step Lanczos on H_q from
 * the node's unit vector e_q (classical Gram-Schmidt applied twice, as for the spectral bounds;
 * FP32 vectors in SQ_MIXED), the eigenvalues theta_qi and squared first eigenvector components
 * w_qi of its tridiagonal (k-point Gauss quadrature of e_q's spectral measure, exact for
 * polynomials of degree <= 2k - 1); rho_q = (2/|dOmega|) sum_i w_qi g(theta_qi) with the Fermi
 * level from 2 sum_q sum_i w_qi g(theta_qi) = N_e (the bisection rule of sq_fermi_level) and
 * E_band = 2 sum_q sum_i w_qi theta_qi g(theta_qi). Independent of sq_moments (it neither needs
 * nor changes the Chebyshev moments; it rebuilds the per-wave lists). k in 1..128 (capped at
 * the region dimension). Host outputs: mu_out, rho_out [N_d] (x fastest), e_band_out, each may
 * be NULL. Allocates and frees its own device scratch, not counted by sq_footprint_bytes: Krylov
 * waves of at most 16 GiB (and at most 80 % of the free device memory; fewer tiles per wave when
 * less is free) plus 2 N_d k + N_d doubles for the Gauss nodes, weights and density; synchronises
 * the stream.
 * Errors: SQ_ERR_INVALID_ARG (k), SQ_ERR_OOM, SQ_ERR_NO_BRACKET, SQ_ERR_CUDA. */
int sq_gauss_density(sq_handle* h, int k, double* mu_out, double* rho_out, double* e_band_out);

/* Green-Kubo shear viscosity (Sec. 5.2, Eq. viscosity) of a stress time series, e.g. the sigma
 * of successive snapshots of a trajectory served through sq_server_*:
 *   eta(k dt) = |Omega| / kT * int_0^{k dt} (1/5) sum_i <s_i(t') s_i(0)> dt',
 *   s_i = sigma_12, sigma_23, sigma_31, (sigma_11 - sigma_22)/2, (sigma_22 - sigma_33)/2.
 * <s_i(k dt) s_i(0)> is the mean of s_i(t + k) s_i(t) over every time origin t = 0..n_steps-1-k
 * of every trajectory (independent initial conditions); the integral is the trapezoid rule.
 * sigma_host: [n_traj][n_steps][9] row-major 3 x 3 stresses (Ha/bohr^3), host memory, not
 * retained. dt: sampling interval (atomic time units, 2.4189e-17 s); volume |Omega| (bohr^3);
 * kT (Ha). Outputs (host): eta_out [max_lag + 1] in atomic units (1 = 0.7117 mPa s),
 * acf_out [max_lag + 1] (Ha^2/bohr^6) or NULL. Runs on the current device on stream (NULL =
 * default) with scratch it allocates and frees; synchronises the stream. Deterministic.
 * Errors: SQ_ERR_INVALID_ARG (NULL sigma_host / eta_out, n_traj < 1, n_steps < 2,
 * max_lag outside [0, n_steps), non-positive dt, volume or kT), SQ_ERR_OOM, SQ_ERR_CUDA; the
 * text is in sq_last_error(NULL). */
int sq_green_kubo(const double* sigma_host, int n_traj, int n_steps, double dt, double volume, double kT,
                  int max_lag, void* stream, double* eta_out, double* acf_out);

void sq_destroy(sq_handle* h);

/* Last error text of h (or of the last failed sq_setup when h is NULL); never NULL. */
const char* sq_last_error(const sq_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* SQ_API_H */
