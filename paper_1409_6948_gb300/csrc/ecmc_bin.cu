// ecmc_bin.cu -- per-sweep draws, cell binning into fixed-capacity buckets,
// the end-of-sweep reduction, and the gather back to disk-id order, for all
// replicas of a handle at once.
//
// Sec. 3.4 steps 1-3: every sweep decomposes the box into cells on a square
// lattice shifted by a random vector and draws one colour order for all
// 2x2 blocks.  A disk belongs to the cell holding its centre.
#include "ecmc_device.cuh"
#include "ecmc_internal.cuh"

namespace ecmc {

// One thread per replica: shift and colour order of sweep state->t from
// Philox(t, 0, 0, 0) under the replica's key.
__global__ void k_sweep_begin(const Geom* __restrict__ rg, SweepState* st, int R,
                              unsigned* sched) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r == 0 && sched != nullptr) {
    // persistent sweep: work list from the start, a new epoch, no abort
    sched[0] = 0u;
    sched[1] += 1u;
    sched[2] = 0u;
  }
  if (r >= R) return;
  const Geom& g = rg[r];
  SweepState& s = st[r];
  const int64_t t = s.t;
  U64x4 u = philox((uint64_t)t, kPurposeSweep, 0, 0, g.seed, g.replica);
  s.sx = unit_double(u.v[0]) * g.w;
  s.sy = unit_double(u.v[1]) * g.h;
  // colour order: permutation number floor(u2 * 24 / 2^64) of (0,1,2,3) in
  // lexicographic order, decoded from its factorial-base digits 6, 2, 1
  int code = (int)below_n(u.v[2], 24);
  int pool[4] = {0, 1, 2, 3};
  const int radix[3] = {6, 2, 1};
  int left = 4;
  for (int i = 0; i < 3; ++i) {
    int d = code / radix[i];
    code -= d * radix[i];
    s.perm[i] = pool[d];
    for (int j = d; j < left - 1; ++j) pool[j] = pool[j + 1];
    --left;
  }
  s.perm[3] = pool[0];
  // axis chains alternate x (even sweeps) and y; isotropic chains use the
  // frame coordinates in (x, y) order
  s.axis = g.dir_mode == 2 ? 0 : (int)(t & 1);
}

void launch_sweep_begin(const DevBufs& b, cudaStream_t s) {
  k_sweep_begin<<<(b.R + 31) / 32, 32, 0, s>>>(b.rg, b.state, b.R, b.sched);
}

// Cell index along one axis as cell_1d computes it in FP64, first estimated
// in FP32 (inputs rounded toward zero on the integer pipes): when the
// estimate's error interval [q - eq, q + eq] holds no cell boundary and lies
// inside (0, cells), its floor is the FP64 result; otherwise (about 2 eq of
// the disks) the FP64 formula runs.
__device__ __forceinline__ int cell_1d_screened(double v, double shift, double L, double inv_w,
                                                int cells, float Lf, float inv_wf, float eq) {
  float uf = to_float_trunc(v) - to_float_trunc(shift);
  uf = uf < 0.0f ? uf + Lf : uf;
  const float qf = uf * inv_wf;
  const float lo = qf - eq, hi = qf + eq;
  if (lo > 0.0f && hi < (float)cells) {
    const int ilo = (int)lo, ihi = (int)hi;  // both positive: truncation is floor
    if (ilo == ihi) return ilo;
  }
  return cell_1d(v, shift, L, inv_w, cells);
}

// Append disk (x, y, id) to its bucket in dst.  Called by every lane of the
// warp (valid = false for lanes without a disk): lanes bound for the same
// cell -- a cell's disks reach at most four cells of the shifted grid --
// take consecutive slots with one atomic per group, so the writes coalesce.
// The slot order inside a bucket is immaterial (frames sort members by id).
__device__ __forceinline__ void bin_one(const Geom* __restrict__ rg,
                                        const SweepState* __restrict__ sts, int rep, bool valid,
                                        double x, double y, int id, double* __restrict__ qx,
                                        double* __restrict__ qy, int* __restrict__ qid,
                                        int* __restrict__ cnt_dst, int cap, int* err) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int cn = -1;
  if (valid) {
    const Geom& g = rg[rep];
    const SweepState& st = sts[rep];
    const int cx = cell_1d_screened(x, st.sx, g.L, g.inv_w, g.cells_x, g.Lf, g.inv_wf,
                                    g.bin_eq_x);
    const int cy = cell_1d_screened(y, st.sy, g.L, g.inv_h, g.cells_y, g.Lf, g.inv_hf,
                                    g.bin_eq_y);
    cn = g.cell_off + cy * g.cells_x + cx;
  }
  const unsigned grp = __match_any_sync(FULL, cn);
  const int leader = __ffs(grp) - 1;
  int base = 0;
  if (valid && lane == leader) base = atomicAdd(&cnt_dst[cn], __popc(grp));
  base = __shfl_sync(FULL, base, leader);
  if (!valid) return;
  const int r = base + __popc(grp & ((1u << lane) - 1u));
  if (r >= cap) {
    atomicCAS(err, DEV_OK, DEV_CAPACITY);
    return;
  }
  const int64_t o = (int64_t)cn * cap + r;
  qx[o] = x;
  qy[o] = y;
  qid[o] = id;
}

// Bin every disk of buffer src into the buckets of buffer dst (whose counts
// are zero on entry).  Bucketed input: thread per slot of the padded array.
__global__ void k_bin_bucketed(const Geom* __restrict__ rg, const SweepState* __restrict__ st,
                               const int* __restrict__ cell_rep, int C_total, int cap,
                               const double* __restrict__ px, const double* __restrict__ py,
                               const int* __restrict__ pid, const int* __restrict__ cnt_src,
                               double* __restrict__ qx, double* __restrict__ qy,
                               int* __restrict__ qid, int* __restrict__ cnt_dst, int* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = i < (int64_t)C_total * cap;  // whole warps reach bin_one
  const int c = in ? (int)(i / cap) : 0;
  const int k = in ? (int)(i - (int64_t)c * cap) : 0;
  const bool valid = in && k < min(__ldg(&cnt_src[c]), cap);
  const int r = valid ? cell_rep[c] : 0;
  bin_one(rg, st, r, valid, valid ? px[i] : 0.0, valid ? py[i] : 0.0, valid ? pid[i] : 0, qx,
          qy, qid, cnt_dst, cap, err);
}

__device__ __forceinline__ int replica_of_disk(const int64_t* __restrict__ n_off, int R,
                                               int64_t i) {
  int lo = 0, hi = R - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (n_off[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Flat input (positions of all replicas concatenated in id order, slots
// 0..N_total-1 of px, py).
__global__ void k_bin_flat(const Geom* __restrict__ rg, const SweepState* __restrict__ st,
                           const int64_t* __restrict__ n_off, int R, int64_t N_total, int cap,
                           const double* __restrict__ px, const double* __restrict__ py,
                           double* __restrict__ qx, double* __restrict__ qy, int* __restrict__ qid,
                           int* __restrict__ cnt_dst, int* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < N_total;  // whole warps reach bin_one
  const int r = valid ? replica_of_disk(n_off, R, i) : 0;
  bin_one(rg, st, r, valid, valid ? px[i] : 0.0, valid ? py[i] : 0.0,
          valid ? (int)(i - n_off[r]) : 0, qx, qy, qid, cnt_dst, cap, err);
}

void launch_bin(const DevBufs& b, int src, int dst, cudaStream_t s) {
  cudaMemsetAsync(b.count[dst], 0, sizeof(int) * (size_t)b.C_total, s);
  const int bs = 256;
  if (src < 0) {  // flat input lives in buffer 1-dst
    const int sb = 1 - dst;
    const int64_t nb = (b.N_total + bs - 1) / bs;
    k_bin_flat<<<(unsigned)nb, bs, 0, s>>>(b.rg, b.state, b.n_off, b.R, b.N_total, b.cap, b.px[sb],
                                          b.py[sb], b.px[dst], b.py[dst], b.pid[dst],
                                          b.count[dst], b.err);
  } else {
    const int64_t total = (int64_t)b.C_total * b.cap;
    const int64_t nb = (total + bs - 1) / bs;
    k_bin_bucketed<<<(unsigned)nb, bs, 0, s>>>(b.rg, b.state, b.cell_rep, b.C_total, b.cap,
                                              b.px[src], b.py[src], b.pid[src], b.count[src],
                                              b.px[dst], b.py[dst], b.pid[dst], b.count[dst],
                                              b.err);
  }
}

// Wrap caller positions (interleaved, id order, replicas concatenated) into
// [0, L) of their replica as a flat list.
__global__ void k_load_flat(const Geom* __restrict__ rg, const int64_t* __restrict__ n_off, int R,
                            int64_t N_total, const double* __restrict__ xy,
                            double* __restrict__ px, double* __restrict__ py) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N_total) return;
  const double L = rg[replica_of_disk(n_off, R, i)].L;
  double x = xy[2 * i], y = xy[2 * i + 1];
  x = x - L * floor(x / L);
  y = y - L * floor(y / L);
  if (x >= L) x -= L;
  if (y >= L) y -= L;
  px[i] = x;
  py[i] = y;
}

void launch_load_flat(const DevBufs& b, const double* xy_dev, cudaStream_t s) {
  const int bs = 256;
  const int other = 1 - b.cur;
  k_load_flat<<<(unsigned)((b.N_total + bs - 1) / bs), bs, 0, s>>>(
      b.rg, b.n_off, b.R, b.N_total, xy_dev, b.px[other], b.py[other]);
}

// Positions back to id order (interleaved pairs, replicas concatenated).
__global__ void k_gather(const Geom* __restrict__ rg, const int* __restrict__ cell_rep,
                         int C_total, int cap, const double* __restrict__ px,
                         const double* __restrict__ py, const int* __restrict__ pid,
                         const int* __restrict__ cnt, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)C_total * cap) return;
  const int c = (int)(i / cap);
  const int k = (int)(i - (int64_t)c * cap);
  if (k >= min(cnt[c], cap)) return;
  const int64_t id = rg[cell_rep[c]].n_off + pid[i];
  out[2 * id] = px[i];
  out[2 * id + 1] = py[i];
}

void launch_gather(const DevBufs& b, double* xy_out, cudaStream_t s) {
  const int bs = 256;
  const int64_t total = (int64_t)b.C_total * b.cap;
  k_gather<<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(
      b.rg, b.cell_rep, b.C_total, b.cap, b.px[b.cur], b.py[b.cur], b.pid[b.cur], b.count[b.cur],
      xy_out);
}

// Local cell of every disk of one replica (by id) in the last binning.
__global__ void k_cells_of(Geom g, int cap, const int* __restrict__ pid,
                           const int* __restrict__ cnt, int* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)g.ncell * cap) return;
  const int lc = (int)(i / cap);
  const int k = (int)(i - (int64_t)lc * cap);
  const int c = g.cell_off + lc;
  if (k >= min(cnt[c], cap)) return;
  out[pid[(int64_t)c * cap + k]] = lc;
}

void launch_cells_of(const Geom& g, const DevBufs& b, int* cell_of_id, cudaStream_t s) {
  const int bs = 256;
  const int64_t total = (int64_t)g.ncell * b.cap;
  k_cells_of<<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(g, b.cap, b.pid[b.cur],
                                                             b.count[b.cur], cell_of_id);
}

// End of sweep, one block per replica: reduce the replica's per-cell results
// in a fixed order (deterministic), add them to its running totals, append
// its member-weighted pressure sums of this sweep to its history, advance its
// sweep counter.
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Partial sums over one chunk of cells (one block per chunk), in a fixed
// order: thread-strided sums, then warp and block trees.
__global__ void __launch_bounds__(256) k_sweep_partials(const CellStats* __restrict__ cs,
                                                        const int2* __restrict__ chunks,
                                                        ChunkSums* __restrict__ out) {
  constexpr int NV = 9;
  __shared__ double sd[2][8];
  __shared__ long long sl[NV][8];
  const int2 ch = chunks[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double b = 0.0, bw = 0.0;
  long long v[NV] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int c = ch.x + tid; c < ch.y; c += blockDim.x) {
    const CellStats s = cs[c];
    b += s.sum_b;
    bw += (double)s.n_mem * s.sum_b;
    v[0] += s.events;
    v[1] += s.lifts;
    v[2] += s.frozen;
    v[3] += s.walls;
    v[4] += s.fp64_evals;
    v[5] += s.chains;
    v[6] += s.replayed;
    v[7] += s.rejected;
    v[8] += (long long)s.n_mem * s.rejected;
  }
  b = warp_sum_d(b);
  bw = warp_sum_d(bw);
  for (int q = 0; q < NV; ++q) v[q] = warp_sum_ll(v[q]);
  if (lane == 0) {
    sd[0][wid] = b;
    sd[1][wid] = bw;
    for (int q = 0; q < NV; ++q) sl[q][wid] = v[q];
  }
  __syncthreads();
  if (tid == 0) {
    ChunkSums r;
    r.sum_b = 0.0;
    r.sum_b_w = 0.0;
    for (int q = 0; q < NV; ++q) r.v[q] = 0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) {
      r.sum_b += sd[0][wv];
      r.sum_b_w += sd[1][wv];
      for (int q = 0; q < NV; ++q) r.v[q] += sl[q][wv];
    }
    out[blockIdx.x] = r;
  }
}

void launch_sweep_partials(const DevBufs& b, cudaStream_t s) {
  k_sweep_partials<<<b.n_chunks, 256, 0, s>>>(b.cell_stats, b.chunks, b.partials);
}

// End of sweep, one thread per replica: add the replica's chunk sums in
// chunk order (deterministic) to its running totals, append its
// member-weighted pressure sums of this sweep to its history, advance its
// sweep counter.
__global__ void k_sweep_end(const Geom* __restrict__ rg, SweepState* st,
                            const ChunkSums* __restrict__ part, const int* __restrict__ chunk_off,
                            RunTotals* tot, double* history, int64_t history_cap, int R) {
  const int rep = blockIdx.x * blockDim.x + threadIdx.x;
  if (rep >= R) return;
  const Geom& g = rg[rep];
  double b = 0.0, bw = 0.0;
  long long v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = chunk_off[rep]; k < chunk_off[rep + 1]; ++k) {
    b += part[k].sum_b;
    bw += part[k].sum_b_w;
    for (int q = 0; q < 9; ++q) v[q] += part[k].v[q];
  }
  RunTotals& T = tot[rep];
  SweepState& S = st[rep];
  // displacement of the accepted chains, each weighted by its cell's members
  const double disp_w = (double)(g.N * (long long)g.n_m - v[8]) * g.ell;
  T.sum_b += b;
  T.sum_b_w += bw;
  T.sum_disp += (double)(v[5] - v[7]) * g.ell;
  T.sum_disp_w += disp_w;
  T.events += v[0];
  T.lifts += v[1];
  T.frozen += v[2];
  T.walls += v[3];
  T.fp64_evals += v[4];
  T.chains += v[5];
  T.replayed += v[6];
  T.rejected += v[7];
  T.sweeps += 1;
  if (history != nullptr && S.history_len < history_cap) {
    double* h = history + 2 * ((int64_t)rep * history_cap + S.history_len);
    h[0] = bw;
    h[1] = disp_w;
  }
  S.history_len += 1;
  S.t += 1;
}

void launch_sweep_end(const DevBufs& b, cudaStream_t s) {
  launch_sweep_partials(b, s);
  k_sweep_end<<<(b.R + 31) / 32, 32, 0, s>>>(b.rg, b.state, b.partials, b.chunk_off, b.totals,
                                             b.history, b.history_cap, b.R);
}

}  // namespace ecmc
