// ecmc_internal.cuh -- shared declarations of the CUDA implementation of the
// parallel event-chain sweep (Kampmann, Boltz, Kierfeld, arXiv:1409.6948).
//
// Data layout in device memory (all per handle):
//   - positions live in "cell buckets": cell c owns the slot range
//     [c * cap_mem, c * cap_mem + count[c]) of the SoA arrays px, py (float64)
//     and pid (int32).  cap_mem is a rigorous bound on the number of disk
//     centres that fit in one cell (disjoint disks of diameter sigma), so the
//     binning pass needs no prefix sum;
//   - two such buffers are used alternately: each sweep bins from one into
//     the other (Sec. 3.4 step 1, new shifted decomposition);
//   - per sweep, the four colour phases (Sec. 3.4 steps 2-6) each run a frame
//     builder, which stages every active cell plus its frozen halo into a
//     fixed-size record, and the chain kernel, which copies that record into
//     shared memory and runs the chains;
//   - a small device struct holds the sweep counter and the per-sweep draws,
//     so one sweep is a fixed sequence of launches (graph-capturable).
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "ecmc.h"

namespace ecmc {

// ---- error word (device) ------------------------------------------------
enum DevErr : int {
  DEV_OK = 0,
  DEV_CAPACITY = 1,   // a bucket or frame record overflowed its rigorous bound
  DEV_CHAIN_CAP = 2,  // a chain reached the per-chain event cap
  DEV_OVERLAP = 3,
  DEV_WAIT_TIMEOUT = 4,  // a dependency wait of the persistent sweep kernel gave up
};

constexpr int64_t kMaxEventsPerChain = int64_t(1) << 22;
// Default width of the candidate strips across the chain axis, in sigma.
constexpr double kDefaultStripWidth = 0.5;
constexpr uint64_t kPurposeSweep = 0, kPurposeChain = 1, kPurposeShuffle = 2;

// ---- per-sweep device state ------------------------------------------------
struct SweepState {
  int64_t t;        // Philox counter of the current sweep
  double sx, sy;    // shift of the cell lattice
  int perm[4];      // colour order
  int axis;         // 0: chains along x, 1: along y
  int flat_input;   // 1: current positions are a flat id-ordered list
  int64_t history_len;
};

// Per-cell results of one sweep (written by the cell's phase).
struct CellStats {
  double sum_b;     // contact sum of the cell's chains, in chain order
  int events, lifts, frozen, walls;
  int fp64_evals, chains, n_mem, replayed;
  int rejected;     // chains rejected under the rejecting boundary rule
};

// Partial sums of one chunk of a replica's cells (end-of-sweep reduction).
struct ChunkSums {
  double sum_b, sum_b_w;
  long long v[9];  // events, lifts, frozen, walls, fp64_evals, chains, replayed,
                   // rejected, sum of n_mem * rejected
};

// Running totals (device).
struct RunTotals {
  double sum_b, sum_disp, sum_b_w, sum_disp_w;
  long long sweeps, chains, events, lifts, frozen, walls, fp64_evals, replayed, rejected;
};

struct ChainRec {
  long long start_id, end_id, events, walls;
};

// ---- static geometry and capacities of one replica -------------------------
// Undo log of one chain under the rejecting boundary rule: every disk that
// became the mover, with its frame coordinates and touched flag before it
// moved.  A straight chain without reflections passes no disk twice (each
// new mover lies ahead of the previous one along d), so a cell needs at most
// one entry per member.
struct UndoEntry {
  double a, b;
  float a32, b32;
  int m, touched;
};

// A handle holds R independent replicas (R = 1 for ecmc_create).  Their cells
// are numbered globally: replica r owns cells [cell_off, cell_off + ncell) and,
// in every colour phase, active cells [act_off, act_off + nact).  All cell
// buckets have the same capacity (the largest over the replicas).
struct Geom {
  int64_t n_off;     // first disk of this replica in concatenated positions
  int cell_off;      // first global cell of this replica
  int act_off;       // first global active cell (per colour phase)
  int nact;          // active cells per colour phase: (cells_x/2)(cells_y/2)
  int rep;           // replica index within the handle
  int64_t N;
  double L, sigma, sig2, w, h, inv_w, inv_h, ell;
  int cells_x, cells_y, ncell;
  int n_m;
  int dir_mode;
  int list_mode;     // 0 start disks drawn with replacement, 1 a shuffled list (negative control)
  uint64_t seed, replica;
  int cap_mem;       // slots per cell bucket (members)
  int cap_obj;       // objects per frame (members + frozen images)
  int nbin;          // strip bins across the chain axis per frame
  float bin_w;       // strip bin width (sigma units already applied)
  float inv_bin_w;
  float sigf;        // sigma as float
  float eps_d;       // bound on |FP32 difference - FP64 difference| in a frame
  float s_margin;    // bound on |FP32 hit distance estimate - FP64 hit distance|
  float sig_plus;    // FP32 miss threshold on |perpendicular offset|
  float sig_minus;   // FP32 certain-hit threshold on |perpendicular offset|
  float sig2f;
  float strip_margin;
  // FP32 screening of isotropic chains (general directions)
  float iso_e;       // bound on |FP32 - FP64| of the projections b = D.d and c = D x d
  float iso_sq;      // bound on the error of the FP32 square root of sigma^2 - c^2
  float iso_r;       // FP32 rounding of the hit-distance bounds
  float iso_sig_lo;  // certain-hit threshold on |c| (below sigma)
  float iso_sig_hi;  // certain-miss threshold on |c| (above sigma)
  int precision;     // 0 FP64 candidates, 1 FP32 screening
  // FP32 cell index of the binning pass: q = (v - s mod L) / w estimated in
  // FP32 within bin_eq_* of the FP64 product; the FP64 formula decides only
  // when that interval touches a cell boundary
  float Lf, inv_wf, inv_hf, bin_eq_x, bin_eq_y;
  int boundary;      // 0 reflect at walls and frozen disks, 1 reject the whole chain
  UndoEntry* undo;   // boundary 1: undo logs, undo_stride entries per global cell
  int undo_stride;   // largest bucket capacity of the handle (>= cap_mem)
};

// Frame record layout of one group of cpw cells (all arrays [index][cpw]).
// The first light_bytes (header, strips, members, FP32 coordinates, keys)
// are what the chain kernel scans; the FP64 coordinates follow, so that the
// kernel may keep only the light part in shared memory.
struct RecLayout {
  int cpw;
  int nbin, cap_mem, cap_obj;
  size_t off_hdr, off_bstart, off_mrank, off_mslot, off_a32, off_b32, off_a64, off_b64,
      off_key, off_info, light_bytes, bytes;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

inline RecLayout make_layout(int cpw, int nbin, int cap_mem, int cap_obj) {
  RecLayout r;
  r.cpw = cpw;
  r.nbin = nbin;
  r.cap_mem = cap_mem;
  r.cap_obj = cap_obj;
  size_t o = 0;
  r.off_hdr = o;     o = align16(o + sizeof(int) * 2 * cpw);
  r.off_bstart = o;  o = align16(o + sizeof(int) * (size_t)(nbin + 1) * cpw);
  r.off_mrank = o;   o = align16(o + sizeof(int) * (size_t)cap_mem * cpw);
  r.off_mslot = o;   o = align16(o + sizeof(int) * (size_t)cap_mem * cpw);
  r.off_a32 = o;     o = align16(o + sizeof(float) * (size_t)cap_obj * cpw);
  r.off_b32 = o;     o = align16(o + sizeof(float) * (size_t)cap_obj * cpw);
  r.off_key = o;     o = align16(o + sizeof(int) * (size_t)cap_obj * cpw);
  r.off_info = o;    o = align16(o + sizeof(int) * (size_t)cap_obj * cpw);
  r.light_bytes = o;
  r.off_a64 = o;     o = align16(o + sizeof(double) * (size_t)cap_obj * cpw);
  r.off_b64 = o;     o = align16(o + sizeof(double) * (size_t)cap_obj * cpw);
  r.bytes = o;
  return r;
}

// Device pointers of one handle (and the host-side sizes launches need).
struct DevBufs {
  double* px[2];
  double* py[2];
  int* pid[2];
  int* count[2];
  int cur;  // buffer holding the current positions
  SweepState* state;       // [R]
  CellStats* cell_stats;   // [C_total]
  RunTotals* totals;       // [R]
  double* history;         // [R][history_cap] pairs: sum_b_w, sum_disp_w
  int64_t history_cap;
  unsigned char* records;  // frame records of one colour
  unsigned char* gtouch;   // touched flags in global memory (fmode 2)
  int fmode;               // where the chain kernel keeps the frames (see phase_smem_bytes)
  unsigned char* stage;    // non-null: frame builder stages objects in global memory
  size_t stage_bytes;      // per active cell
  int* err;
  ChainRec* chain_recs;    // optional, [C_total * max n_m]
  int rec_stride;          // chain records per cell
  const Geom* rg;          // [R] device copy of the replicas' geometry
  const int* cell_rep;     // [C_total] replica of every global cell
  const int* act_rep;      // [A_total] replica of every global active cell
  const int64_t* n_off;    // [R + 1] disk offsets
  const int2* chunks;      // [n_chunks] (first, last+1) global cells, replica-aligned
  const int* chunk_off;    // [R + 1] first chunk of every replica
  ChunkSums* partials;     // [n_chunks]
  int n_chunks;
  int replay;              // 1 = replay repeating reflection legs (chain kernel)
  int iso;                 // 1 = isotropic directions
  int reject;              // 1 = rejecting boundary rule (axis chains)
  unsigned* sched;         // persistent sweep: [0] next work item, [1] epoch, [2] abort
  unsigned* done;          // [C_total] epoch in which each cell last finished
  unsigned long long wait_ns;  // limit of one dependency wait
  int wait_test;           // 1 = dependency waits look for a value nobody writes
  int R, C_total, A_total, cap;
  int64_t N_total;
};

// ---- launchers (defined in the .cu files) --------------------------------
// Every launcher covers all replicas of the handle, except the measurements
// (min_dist, gr, cells_of), which take the replica's host-side geometry.
void launch_sweep_begin(const DevBufs& b, cudaStream_t s);
void launch_bin(const DevBufs& b, int src, int dst, cudaStream_t s);
void launch_frame_build(const DevBufs& b, const RecLayout& lay, int colour_index,
                        cudaStream_t s);
int launch_phase(const DevBufs& b, const RecLayout& lay, int colour_index, int tpc,
                 int warps_per_block, int records_on, int precision, cudaStream_t s);
void launch_sweep_partials(const DevBufs& b, cudaStream_t s);
void launch_sweep_end(const DevBufs& b, cudaStream_t s);
void launch_gather(const DevBufs& b, double* xy_out, cudaStream_t s);
void launch_load_flat(const DevBufs& b, const double* xy_dev, cudaStream_t s);
void launch_cells_of(const Geom& g, const DevBufs& b, int* cell_of_id, cudaStream_t s);
int launch_hexatic(const DevBufs& b, double rs, double2* psi_k, int* nn,
                   unsigned long long* bad, cudaStream_t s);
void launch_min_dist(const Geom& g, const DevBufs& b, double rcut, unsigned long long* out,
                     cudaStream_t s);
void launch_gr(const Geom& g, const DevBufs& b, double dr, int nbins, unsigned long long* counts,
               cudaStream_t s);
size_t frame_build_smem(const RecLayout& lay);
size_t frame_stage_bytes(const RecLayout& lay);
int configure_frame_build(const RecLayout& lay);
int configure_phase(const RecLayout& lay, int tpc, int warps, int fmode);
int probe_peaks(double* smem_gbs, double* fp64_gflops);
size_t fused_smem_bytes(const RecLayout& lay, int fm);
size_t fused_scratch_bytes(const RecLayout& lay);
// Chain-loop variant of the kernels: 0 axis chains reflected at walls and
// frozen disks, 1 isotropic chains, 2 axis chains under the rejecting
// boundary rule (a compile-time variant, so that the default loop carries
// none of its bookkeeping).
// Set the message ecmc_last_error_message() returns; returns code.
int report_error(int code, const char* msg);

// The FP32 binning screen of replica g (host).  With v, s rounded toward
// zero to FP32 (relative error 2^-23) and each FP32 operation rounded
// (2^-24), |u32 - u| <= 2^-21 (L + w) after the wrap, so the FP32 quotient
// is within 2^-21 (L + w) / w + 2^-23 cells of the FP64 product; bin_eq_*
// is twice that.
inline void set_bin_screen(Geom& g) {
  g.Lf = (float)g.L;
  g.inv_wf = (float)g.inv_w;
  g.inv_hf = (float)g.inv_h;
  g.bin_eq_x = (float)(2.0 * (std::ldexp(1.0, -21) * (g.L + g.w) * g.inv_w * 1.01 +
                              std::ldexp(1.0, -23) * g.cells_x));
  g.bin_eq_y = (float)(2.0 * (std::ldexp(1.0, -21) * (g.L + g.h) * g.inv_h * 1.01 +
                              std::ldexp(1.0, -23) * g.cells_y));
}

// Shared by the handle path and the allocation-free entry point
// (ecmc_api.cu): argument checks, geometry, bucket and frame capacities and
// n_m of one replica (returns ECMC_OK or ECMC_ERR_ARG with the message set;
// lattice_start = 1 also requires N to be a perfect square whose square
// lattice does not overlap); the FP32 screening bounds of the chain kernel;
// the strips across the chain axis, strip_w in units of sigma.
int setup_replica_geom(const ecmc_replica_desc_t& d, Geom& g, int lattice_start);
void set_screen_bounds(Geom& g);
void set_strip_bins(Geom& g, double strip_w);

inline int chain_kind(const DevBufs& b) { return b.iso ? 1 : (b.reject ? 2 : 0); }
int configure_fused(const RecLayout& lay, int tpc, int fm, int kind, int* blocks_per_sm);
int launch_fused(const DevBufs& b, const RecLayout& lay, int tpc, int blocks, int records_on,
                 int precision, cudaStream_t s);
int launch_sqrt_rn(const double* x, double* out, int64_t n, cudaStream_t s);
void host_sqrt_rn(const double* x, double* out, int64_t n, double rel_error);
// fmode: 0 = whole frame in shared memory, 1 = FP64 coordinates in global
// memory, 2 = whole frame in global memory
size_t phase_smem_bytes(const RecLayout& lay, int warps_per_block, int fmode = 0);
int phase_max_warps(const RecLayout& lay, int tpc);

}  // namespace ecmc
