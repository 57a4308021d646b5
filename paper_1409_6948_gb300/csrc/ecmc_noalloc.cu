// ecmc_noalloc.cu -- ecmc_sweep_noalloc: sweeps of a caller-held system
// without any device allocation.
//
// Some callers cannot allocate device memory: an application whose device
// memory is owned by its own pool (every cudaMalloc outside it is forbidden),
// or code that must not allocate once its set-up phase is over.  This entry
// point runs the same kernels as ecmc_sweep, but all of its scratch memory
// (cell buckets, frame records, per-cell results, sweep state) is carved out
// of one file-scope __device__ array of ECMC_NOALLOC_SCRATCH_BYTES bytes that
// is part of the library image: every GPU that loads the library holds it
// until the process exits.  The caller passes the positions (device memory,
// read and overwritten) and the system's parameters.
//
// The array is shared by every call: calls that overlap on the GPU (on
// different streams, or from different host threads) race on it and must be
// serialised by the caller.  What must start at zero (bucket counts,
// running totals, the error word, the overlap check's minimum) is set by
// every call; the rest is written before it is read.
//
// Argument checks, geometry, capacities and the FP32 screening bounds come
// from the same functions the handle path uses (ecmc_api.cu), and the input
// passes the same overlap check as ecmc_set_positions.  On any error the
// caller's positions are left as they were passed in: device errors are read
// before the positions are written back.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ecmc.h"
#include "ecmc_internal.cuh"

using namespace ecmc;

static __device__ __align__(256) unsigned char g_noalloc_scratch[ECMC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// the name g_noalloc_scratch is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.  The
// cache is not invalidated: after cudaDeviceReset the cached address is
// stale, so a process that resets a device must not call this entry point
// on it again.
int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ECMC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
      return ECMC_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return ECMC_OK;
}

size_t carve(size_t& off, size_t bytes) {
  const size_t at = (off + 255) & ~size_t(255);
  off = at + bytes;
  return at;
}

}  // namespace

extern "C" int ecmc_sweep_noalloc(double* xy, int64_t N, double L, double sigma, int cells_x,
                                  int cells_y, double ell, int n_m, uint64_t seed,
                                  uint64_t replica, int64_t t0, int64_t n_sweeps, void* stream) {
  if (!xy) return report_error(ECMC_ERR_ARG, "xy is NULL");
  if (n_m < 1 || t0 < 0 || n_sweeps < 0)
    return report_error(ECMC_ERR_ARG, "n_m must be >= 1, t0 and n_sweeps >= 0");

  // geometry, capacities and screening bounds exactly as for a handle (any
  // N: the caller supplies the positions, no lattice start)
  ecmc_replica_desc_t d;
  std::memset(&d, 0, sizeof(d));
  d.N = N;
  d.L = L;
  d.sigma = sigma;
  d.cells_x = cells_x;
  d.cells_y = cells_y;
  d.ell = ell;
  d.n_m = n_m;
  d.seed = seed;
  d.replica = replica;
  Geom g;
  const int grc = setup_replica_geom(d, g, 0);
  if (grc != ECMC_OK) return grc;
  set_strip_bins(g, kDefaultStripWidth);

  int tpc = 32;
  for (int t = 4; t <= 32; t *= 2) {
    if (phase_smem_bytes(make_layout(32 / t, g.nbin, g.cap_mem, g.cap_obj), 1, 0) <= 52 * 1024) {
      tpc = t;
      break;
    }
  }
  const RecLayout lay = make_layout(32 / tpc, g.nbin, g.cap_mem, g.cap_obj);
  // the handle would fall back to frames in global memory here, which needs
  // scratch beyond what this entry point carves
  if (phase_smem_bytes(lay, 1, 0) > 232448 || frame_build_smem(lay) > 232448)
    return report_error(ECMC_ERR_UNSUPPORTED, "cell frames too large for shared memory");

  // carve the scratch array
  const size_t slots = (size_t)g.ncell * g.cap_mem;
  const int n_active = g.nact;
  const int n_groups = (n_active + lay.cpw - 1) / lay.cpw;
  size_t off = 0;
  size_t o_px[2], o_py[2], o_pid[2], o_cnt[2];
  for (int i = 0; i < 2; ++i) {
    o_px[i] = carve(off, sizeof(double) * slots);
    o_py[i] = carve(off, sizeof(double) * slots);
    o_pid[i] = carve(off, sizeof(int) * slots);
    o_cnt[i] = carve(off, sizeof(int) * (size_t)g.ncell);
  }
  const size_t o_state = carve(off, sizeof(SweepState));
  const size_t o_stats = carve(off, sizeof(CellStats) * (size_t)g.ncell);
  const size_t o_tot = carve(off, sizeof(RunTotals));
  const size_t o_err = carve(off, sizeof(int));
  const size_t o_min = carve(off, sizeof(unsigned long long));
  const size_t o_rec = carve(off, (size_t)n_groups * lay.bytes);
  const size_t o_geo = carve(off, sizeof(Geom));
  const size_t o_crep = carve(off, sizeof(int) * (size_t)g.ncell);
  const size_t o_arep = carve(off, sizeof(int) * (size_t)n_active);
  const size_t o_noff = carve(off, sizeof(int64_t) * 2);
  const int n_chunks = (g.ncell + 2047) / 2048;
  const size_t o_chunks = carve(off, sizeof(int2) * (size_t)n_chunks);
  const size_t o_choff = carve(off, sizeof(int) * 2);
  const size_t o_part = carve(off, sizeof(ChunkSums) * (size_t)n_chunks);
  // larger systems than the static array can serve are rejected up front
  if (off > (size_t)ECMC_NOALLOC_SCRATCH_BYTES)
    return report_error(ECMC_ERR_CAPACITY, "system needs more scratch than the static array");

  unsigned char* base = nullptr;
  if (scratch_address(&base) != ECMC_OK)
    return report_error(ECMC_ERR_CUDA, "device address of the scratch array not available");
  DevBufs b;
  std::memset(&b, 0, sizeof(b));
  b.replay = 1;
  for (int i = 0; i < 2; ++i) {
    b.px[i] = reinterpret_cast<double*>(base + o_px[i]);
    b.py[i] = reinterpret_cast<double*>(base + o_py[i]);
    b.pid[i] = reinterpret_cast<int*>(base + o_pid[i]);
    b.count[i] = reinterpret_cast<int*>(base + o_cnt[i]);
  }
  b.state = reinterpret_cast<SweepState*>(base + o_state);
  b.cell_stats = reinterpret_cast<CellStats*>(base + o_stats);
  b.totals = reinterpret_cast<RunTotals*>(base + o_tot);
  b.err = reinterpret_cast<int*>(base + o_err);
  unsigned long long* d_min = reinterpret_cast<unsigned long long*>(base + o_min);
  b.records = base + o_rec;
  b.history = nullptr;
  b.history_cap = 0;
  b.chain_recs = nullptr;
  b.rec_stride = n_m;
  b.cur = 0;
  b.rg = reinterpret_cast<Geom*>(base + o_geo);
  b.cell_rep = reinterpret_cast<int*>(base + o_crep);
  b.act_rep = reinterpret_cast<int*>(base + o_arep);
  b.n_off = reinterpret_cast<int64_t*>(base + o_noff);
  b.R = 1;
  b.C_total = g.ncell;
  b.A_total = n_active;
  b.cap = g.cap_mem;
  b.N_total = N;
  b.chunks = reinterpret_cast<int2*>(base + o_chunks);
  b.chunk_off = reinterpret_cast<int*>(base + o_choff);
  b.partials = reinterpret_cast<ChunkSums*>(base + o_part);
  b.n_chunks = n_chunks;
  b.fmode = 0;
  const int64_t n_off_host[2] = {0, N};
  const int chunk_off_host[2] = {0, n_chunks};
  // the overlap check's running minimum starts at (2 sigma)^2, the cut-off
  const double r2 = 4.0 * g.sig2;
  unsigned long long r2_bits = 0;
  std::memcpy(&r2_bits, &r2, sizeof(r2));

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (configure_frame_build(lay) || configure_phase(lay, tpc, 1, 0))
    return report_error(ECMC_ERR_CUDA, "kernel configuration failed");

  // clear what must start at zero, set the sweep counter
  SweepState st;
  std::memset(&st, 0, sizeof(st));
  st.t = t0;
  if (cudaMemsetAsync(b.count[0], 0, sizeof(int) * (size_t)g.ncell, s) != cudaSuccess ||
      cudaMemsetAsync(b.count[1], 0, sizeof(int) * (size_t)g.ncell, s) != cudaSuccess ||
      cudaMemsetAsync(b.totals, 0, sizeof(RunTotals), s) != cudaSuccess ||
      cudaMemsetAsync(b.err, 0, sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync((void*)b.cell_rep, 0, sizeof(int) * (size_t)g.ncell, s) != cudaSuccess ||
      cudaMemsetAsync((void*)b.act_rep, 0, sizeof(int) * (size_t)n_active, s) != cudaSuccess ||
      cudaMemcpyAsync((void*)b.rg, &g, sizeof(g), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync((void*)b.n_off, n_off_host, sizeof(n_off_host), cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      cudaMemcpyAsync(b.state, &st, sizeof(st), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_min, &r2_bits, sizeof(r2_bits), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync((void*)b.chunk_off, chunk_off_host, sizeof(chunk_off_host),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return report_error(ECMC_ERR_CUDA, "scratch initialisation failed");
  for (int k = 0; k < n_chunks; ++k) {
    const int2 ch = make_int2(k * 2048, (k + 1) * 2048 < g.ncell ? (k + 1) * 2048 : g.ncell);
    if (cudaMemcpyAsync((void*)(b.chunks + k), &ch, sizeof(ch), cudaMemcpyHostToDevice, s) !=
        cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      return report_error(ECMC_ERR_CUDA, "scratch initialisation failed");
  }

  // caller positions -> buckets; then the overlap check of ecmc_set_positions
  // (its fixed-point copy lives in the second bucket buffer, free until the
  // first sweep)
  launch_load_flat(b, xy, s);
  launch_sweep_begin(b, s);
  launch_bin(b, -1, b.cur, s);
  launch_min_dist(g, b, 2.0 * g.sigma, d_min, s);
  int err = 0;
  unsigned long long min_bits = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&err, b.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&min_bits, d_min, sizeof(min_bits), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return report_error(ECMC_ERR_CUDA, "loading the positions failed");
  if (err == DEV_CAPACITY)
    return report_error(ECMC_ERR_CAPACITY, "a cell bucket exceeded its packing bound (overlap)");
  if (err != DEV_OK) return report_error(ECMC_ERR_CUDA, "device error while loading positions");
  double d2 = 0.0;
  std::memcpy(&d2, &min_bits, sizeof(d2));
  if (d2 < g.sig2 * (1.0 - 1e-9))
    return report_error(ECMC_ERR_OVERLAP, "positions overlap: smallest distance below sigma");

  // n sweeps, then the device error word; the positions go back to the
  // caller only if no sweep raised an error
  for (int64_t i = 0; i < n_sweeps; ++i) {
    const int src = b.cur, dst = 1 - b.cur;
    launch_sweep_begin(b, s);
    launch_bin(b, src, dst, s);
    b.cur = dst;
    for (int ci = 0; ci < 4; ++ci) {
      launch_frame_build(b, lay, ci, s);
      if (launch_phase(b, lay, ci, tpc, 1, 0, 1, s))
        return report_error(ECMC_ERR_CUDA, "chain kernel launch failed");
    }
    launch_sweep_end(b, s);
  }
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&err, b.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return report_error(ECMC_ERR_CUDA, "sweep failed");
  if (err == DEV_CAPACITY)
    return report_error(ECMC_ERR_CAPACITY, "a cell bucket or frame exceeded its packing bound");
  if (err == DEV_CHAIN_CAP)
    return report_error(ECMC_ERR_CHAIN_CAP, "a chain reached the per-chain event cap");
  if (err != DEV_OK) return report_error(ECMC_ERR_CUDA, "device error during the sweeps");
  launch_gather(b, xy, s);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return report_error(ECMC_ERR_CUDA, "writing the positions back failed");
  return ECMC_OK;
}
