// ecmc_bin.cu -- per-sweep draws, cell binning into fixed-capacity buckets,
// the end-of-sweep reduction, and the gather back to disk-id order.
//
// Sec. 3.4 steps 1-3: every sweep decomposes the box into cells on a square
// lattice shifted by a random vector and draws one colour order for all
// 2x2 blocks.  A disk belongs to the cell holding its centre.
#include "ecmc_device.cuh"
#include "ecmc_internal.cuh"

namespace ecmc {

// One thread: shift and colour order of sweep state->t from Philox(t, 0, 0, 0).
__global__ void k_sweep_begin(Geom g, SweepState* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int64_t t = st->t;
  U64x4 u = philox((uint64_t)t, kPurposeSweep, 0, 0, g.seed, g.replica);
  st->sx = unit_double(u.v[0]) * g.w;
  st->sy = unit_double(u.v[1]) * g.h;
  // colour order: permutation number floor(u2 * 24 / 2^64) of (0,1,2,3) in
  // lexicographic order, decoded from its factorial-base digits 6, 2, 1
  int code = (int)below_n(u.v[2], 24);
  int pool[4] = {0, 1, 2, 3};
  const int radix[3] = {6, 2, 1};
  int left = 4;
  for (int i = 0; i < 3; ++i) {
    int d = code / radix[i];
    code -= d * radix[i];
    st->perm[i] = pool[d];
    for (int j = d; j < left - 1; ++j) pool[j] = pool[j + 1];
    --left;
  }
  st->perm[3] = pool[0];
  st->axis = (int)(t & 1);
}

void launch_sweep_begin(const Geom& g, const DevBufs& b, cudaStream_t s) {
  k_sweep_begin<<<1, 32, 0, s>>>(g, b.state);
}

// Bin every disk of buffer src into the buckets of buffer dst (whose counts
// are zero on entry).  Bucketed input: thread per slot of the padded array.
__global__ void k_bin_bucketed(Geom g, const SweepState* __restrict__ st,
                               const double* __restrict__ px, const double* __restrict__ py,
                               const int* __restrict__ pid, const int* __restrict__ cnt_src,
                               double* __restrict__ qx, double* __restrict__ qy,
                               int* __restrict__ qid, int* __restrict__ cnt_dst, int* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)g.ncell * g.cap_mem;
  if (i >= total) return;
  const int c = (int)(i / g.cap_mem);
  const int k = (int)(i - (int64_t)c * g.cap_mem);
  if (k >= min(__ldg(&cnt_src[c]), g.cap_mem)) return;
  const double x = px[i], y = py[i];
  const int id = pid[i];
  const double sx = st->sx, sy = st->sy;
  const int cx = cell_1d(x, sx, g.L, g.inv_w, g.cells_x);
  const int cy = cell_1d(y, sy, g.L, g.inv_h, g.cells_y);
  const int cn = cy * g.cells_x + cx;
  const int r = atomicAdd(&cnt_dst[cn], 1);
  if (r >= g.cap_mem) {
    atomicCAS(err, DEV_OK, DEV_CAPACITY);
    return;
  }
  const int64_t o = (int64_t)cn * g.cap_mem + r;
  qx[o] = x;
  qy[o] = y;
  qid[o] = id;
}

// Flat input (positions in id order, slots 0..N-1 of px, py).
__global__ void k_bin_flat(Geom g, const SweepState* __restrict__ st,
                           const double* __restrict__ px, const double* __restrict__ py,
                           double* __restrict__ qx, double* __restrict__ qy, int* __restrict__ qid,
                           int* __restrict__ cnt_dst, int* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  const double x = px[i], y = py[i];
  const int cx = cell_1d(x, st->sx, g.L, g.inv_w, g.cells_x);
  const int cy = cell_1d(y, st->sy, g.L, g.inv_h, g.cells_y);
  const int cn = cy * g.cells_x + cx;
  const int r = atomicAdd(&cnt_dst[cn], 1);
  if (r >= g.cap_mem) {
    atomicCAS(err, DEV_OK, DEV_CAPACITY);
    return;
  }
  const int64_t o = (int64_t)cn * g.cap_mem + r;
  qx[o] = x;
  qy[o] = y;
  qid[o] = (int)i;
}

void launch_bin(const Geom& g, const DevBufs& b, int src, int dst, cudaStream_t s) {
  cudaMemsetAsync(b.count[dst], 0, sizeof(int) * (size_t)g.ncell, s);
  const int bs = 256;
  if (src < 0) {  // flat input lives in buffer 1-dst
    const int sb = 1 - dst;
    const int64_t nb = (g.N + bs - 1) / bs;
    k_bin_flat<<<(unsigned)nb, bs, 0, s>>>(g, b.state, b.px[sb], b.py[sb], b.px[dst], b.py[dst],
                                          b.pid[dst], b.count[dst], b.err);
  } else {
    const int64_t total = (int64_t)g.ncell * g.cap_mem;
    const int64_t nb = (total + bs - 1) / bs;
    k_bin_bucketed<<<(unsigned)nb, bs, 0, s>>>(g, b.state, b.px[src], b.py[src], b.pid[src],
                                              b.count[src], b.px[dst], b.py[dst], b.pid[dst],
                                              b.count[dst], b.err);
  }
}

// Wrap caller positions (interleaved, id order) into [0, L) as a flat list.
__global__ void k_load_flat(Geom g, const double* __restrict__ xy, double* __restrict__ px,
                            double* __restrict__ py) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  double x = xy[2 * i], y = xy[2 * i + 1];
  x = x - g.L * floor(x / g.L);
  y = y - g.L * floor(y / g.L);
  if (x >= g.L) x -= g.L;
  if (y >= g.L) y -= g.L;
  px[i] = x;
  py[i] = y;
}

void launch_load_flat(const Geom& g, const DevBufs& b, const double* xy_dev, cudaStream_t s) {
  const int bs = 256;
  const int other = 1 - b.cur;
  k_load_flat<<<(unsigned)((g.N + bs - 1) / bs), bs, 0, s>>>(g, xy_dev, b.px[other], b.py[other]);
}

// Positions back to id order (interleaved pairs).
__global__ void k_gather(Geom g, const double* __restrict__ px, const double* __restrict__ py,
                         const int* __restrict__ pid, const int* __restrict__ cnt,
                         double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)g.ncell * g.cap_mem;
  if (i >= total) return;
  const int c = (int)(i / g.cap_mem);
  const int k = (int)(i - (int64_t)c * g.cap_mem);
  if (k >= min(cnt[c], g.cap_mem)) return;
  const int id = pid[i];
  out[2 * (int64_t)id] = px[i];
  out[2 * (int64_t)id + 1] = py[i];
}

void launch_gather(const Geom& g, const DevBufs& b, double* xy_out, cudaStream_t s) {
  const int bs = 256;
  const int64_t total = (int64_t)g.ncell * g.cap_mem;
  k_gather<<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(g, b.px[b.cur], b.py[b.cur],
                                                           b.pid[b.cur], b.count[b.cur], xy_out);
}

__global__ void k_cells_of(Geom g, const int* __restrict__ pid, const int* __restrict__ cnt,
                           int* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)g.ncell * g.cap_mem;
  if (i >= total) return;
  const int c = (int)(i / g.cap_mem);
  const int k = (int)(i - (int64_t)c * g.cap_mem);
  if (k >= min(cnt[c], g.cap_mem)) return;
  out[pid[i]] = c;
}

void launch_cells_of(const Geom& g, const DevBufs& b, int* cell_of_id, cudaStream_t s) {
  const int bs = 256;
  const int64_t total = (int64_t)g.ncell * g.cap_mem;
  k_cells_of<<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(g, b.pid[b.cur], b.count[b.cur],
                                                             cell_of_id);
}

// End of sweep: reduce the per-cell results in a fixed order (deterministic),
// add them to the running totals, append the member-weighted pressure sums of
// this sweep to the history, advance the sweep counter.
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(1024) k_sweep_end(Geom g, SweepState* st,
                                                    const CellStats* __restrict__ cs,
                                                    RunTotals* tot, double* history,
                                                    int64_t history_cap) {
  __shared__ double sd[2][32];
  __shared__ long long sl[6][32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double b = 0.0, bw = 0.0;
  long long v[6] = {0, 0, 0, 0, 0, 0};
  for (int c = tid; c < g.ncell; c += blockDim.x) {
    const CellStats s = cs[c];
    b += s.sum_b;
    bw += (double)s.n_mem * s.sum_b;
    v[0] += s.events;
    v[1] += s.lifts;
    v[2] += s.frozen;
    v[3] += s.walls;
    v[4] += s.fp64_evals;
    v[5] += s.chains;
  }
  b = warp_sum_d(b);
  bw = warp_sum_d(bw);
  for (int q = 0; q < 6; ++q) v[q] = warp_sum_ll(v[q]);
  if (lane == 0) {
    sd[0][wid] = b;
    sd[1][wid] = bw;
    for (int q = 0; q < 6; ++q) sl[q][wid] = v[q];
  }
  __syncthreads();
  if (wid != 0) return;
  const int nw = blockDim.x >> 5;
  b = lane < nw ? sd[0][lane] : 0.0;
  bw = lane < nw ? sd[1][lane] : 0.0;
  for (int q = 0; q < 6; ++q) v[q] = lane < nw ? sl[q][lane] : 0;
  b = warp_sum_d(b);
  bw = warp_sum_d(bw);
  for (int q = 0; q < 6; ++q) v[q] = warp_sum_ll(v[q]);
  if (lane == 0) {
    const double disp_w = (double)g.N * (double)g.n_m * g.ell;
    tot->sum_b += b;
    tot->sum_b_w += bw;
    tot->sum_disp += (double)v[5] * g.ell;
    tot->sum_disp_w += disp_w;
    tot->events += v[0];
    tot->lifts += v[1];
    tot->frozen += v[2];
    tot->walls += v[3];
    tot->fp64_evals += v[4];
    tot->chains += v[5];
    tot->sweeps += 1;
    if (st->history_len < history_cap) {
      history[2 * st->history_len] = bw;
      history[2 * st->history_len + 1] = disp_w;
    }
    st->history_len += 1;
    st->t += 1;
  }
}

void launch_sweep_end(const Geom& g, const DevBufs& b, cudaStream_t s) {
  k_sweep_end<<<1, 1024, 0, s>>>(g, b.state, b.cell_stats, b.totals, b.history, b.history_cap);
}

}  // namespace ecmc
