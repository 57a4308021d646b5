// ecmc_sweep.cu -- the persistent sweep kernel: all four colour phases of a
// sweep (Sec. 3.4 steps 4-6) in one launch.
//
// Work list: item i = (colour phase ci, group G) in the order of i = ci * groups + G;
// a group is the cpw = 32/TPC consecutive active cells one warp serves.  Each
// warp takes the next item from a device counter, waits until every
// neighbour cell of an earlier colour phase of the same sweep has finished,
// builds the group's frames in its shared memory, runs the chains (the loop of
// ecmc_chain.cuh) and publishes the cells as finished.  Frozen disks of a later
// colour have not moved yet, and a later cell waits for this one in turn, so
// every cell sees exactly the configuration of the phase-by-phase schedule,
// and the results are those of the per-phase launches bit for bit.  The tail of
// one colour phase overlaps the start of the next.
//
// Progress: an item only waits for items with a smaller index, which were
// taken earlier by running warps and never wait for later items; the
// smallest unfinished item therefore always progresses, whatever the number of
// resident warps.  Every wait is bounded nonetheless (global timer): on
// timeout the kernel raises DEV_WAIT_TIMEOUT and an abort flag that makes
// every warp leave at its next item or wait.
#include "ecmc_build.cuh"
#include "ecmc_chain.cuh"
#include "ecmc_chain_iso.cuh"

namespace ecmc {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned load_volatile(const unsigned* p) {
  return *(const volatile unsigned*)p;
}

// Shared memory of one warp: the frame record of its group, the touched
// flags, the leg histories (which also serve as the builder's staging area,
// used before the chains start) and the builder's scratch.
__host__ __device__ inline size_t fused_touch_bytes(const RecLayout& lay) {
  return align16((size_t)lay.cap_obj * lay.cpw);
}
__host__ __device__ inline size_t fused_hist_bytes(const RecLayout& lay) {
  const size_t h = kHistLegBytes * kHist * (size_t)lay.cpw;
  const size_t s = build_stage_bytes(lay);
  return h > s ? h : s;
}
// FM 0: the whole record in shared memory; FM 1: the FP64 coordinates in a
// per-warp scratch area of global memory (L1/L2), so that more warps fit.
__host__ __device__ inline size_t fused_fp64_bytes(const RecLayout& lay) {
  return lay.bytes - lay.light_bytes;
}
__host__ __device__ inline size_t fused_warp_bytes(const RecLayout& lay, int fm) {
  return (fm == 1 ? lay.light_bytes : lay.bytes) + fused_touch_bytes(lay) +
         fused_hist_bytes(lay) + build_aux_bytes(32);
}

template <int TPC, bool SCREEN, int FM, int KIND = 0>
__global__ void __launch_bounds__(32, 16) k_sweep_fused(
    const Geom* __restrict__ rg, const SweepState* __restrict__ sts,
    const int* __restrict__ act_rep, int n_active, int cap, double* __restrict__ px,
    double* __restrict__ py, const int* __restrict__ pid, const int* __restrict__ cnt,
    RecLayout lay, CellStats* __restrict__ cs, ChainRec* __restrict__ recs, int rec_stride,
    int replay, unsigned* sched, unsigned* done, unsigned long long wait_ns, int wait_test,
    unsigned char* __restrict__ fscratch, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int CPW = 32 / TPC;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned char* const rec = smem;
  unsigned char* const tbase = rec + (FM == 1 ? lay.light_bytes : lay.bytes);
  // the FP64 coordinates: in the record, or in this warp's scratch area
  double* const a64 =
      FM == 1 ? (double*)(fscratch + (size_t)blockIdx.x * fused_fp64_bytes(lay))
              : (double*)(rec + lay.off_a64);
  double* const b64 = a64 + (lay.off_b64 - lay.off_a64) / sizeof(double);
  unsigned char* const hbase = tbase + fused_touch_bytes(lay);
  unsigned char* const aux = hbase + fused_hist_bytes(lay);

  Frame f;
  f.cpw = CPW;
  f.bst = (const int*)(rec + lay.off_bstart);
  f.mrank = (const int*)(rec + lay.off_mrank);
  f.mslot = (const int*)(rec + lay.off_mslot);
  f.a32 = (float*)(rec + lay.off_a32);
  f.b32 = (float*)(rec + lay.off_b32);
  f.a64 = a64;
  f.b64 = b64;
  f.key = (const int*)(rec + lay.off_key);
  f.info = (const int*)(rec + lay.off_info);
  f.touched = tbase;
  const int* hdr = (const int*)(rec + lay.off_hdr);
  LegHist hs;
  hs.P = (double*)hbase;
  hs.step = hs.P + kHist * CPW;
  hs.addb = hs.step + kHist * CPW;
  hs.m = (int*)(hs.addb + kHist * CPW);
  hs.flags = hs.m + kHist * CPW;

  // the sweep's epoch: cells finished in this sweep carry it in done[]; the
  // failure test waits for a value nobody writes
  const unsigned epoch = load_volatile(&sched[1]);
  const unsigned want = wait_test ? (epoch ^ 0x80000000u) : epoch;
  const int n_groups = (n_active + CPW - 1) / CPW;
  const int n_items = 4 * n_groups;
  const int gi = lane / TPC, sub = lane - gi * TPC;

  for (;;) {
    int item = 0;
    if (lane == 0) item = (int)atomicAdd(&sched[0], 1u);
    item = __shfl_sync(FULL, item, 0);
    if (item >= n_items || load_volatile(&sched[2]) != 0u) break;
    const int ci = item / n_groups, G = item - ci * n_groups;

    // this lane group's cell
    const int a = G * CPW + gi;
    const bool valid = a < n_active;
    const int rep = valid ? act_rep[a] : act_rep[n_active - 1];
    const Geom& g = rg[rep];
    const SweepState* st = sts + rep;
    const int colour = st->perm[ci];
    const int hx = g.cells_x >> 1;
    const int la = a - g.act_off;
    const int cx = 2 * (la % hx) + (colour & 1);
    const int cy = 2 * (la / hx) + (colour >> 1);

    // wait for the neighbours of earlier colour phases (lanes of the group
    // share the eight directions)
    bool ok = true;
    if (valid && ci > 0) {
      int phase_of[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) phase_of[st->perm[k]] = k;
      for (int d = sub; d < 8; d += TPC) {
        const int e = d < 4 ? d : d + 1;  // skip the centre of the 3x3 block
        const int ddx = e % 3 - 1, ddy = e / 3 - 1;
        const int ncol = colour ^ (ddx != 0 ? 1 : 0) ^ (ddy != 0 ? 2 : 0);
        if (phase_of[ncol] >= ci) continue;
        int qx = cx + ddx, qy = cy + ddy;
        qx += qx < 0 ? g.cells_x : 0;
        qx -= qx >= g.cells_x ? g.cells_x : 0;
        qy += qy < 0 ? g.cells_y : 0;
        qy -= qy >= g.cells_y ? g.cells_y : 0;
        const int q = g.cell_off + qy * g.cells_x + qx;
        if (load_volatile(&done[q]) == want) continue;
        const unsigned long long t0 = global_ns();
        while (load_volatile(&done[q]) != want) {
          if (load_volatile(&sched[2]) != 0u) {
            ok = false;
            break;
          }
          if (global_ns() - t0 > wait_ns) {
            atomicCAS(err, DEV_OK, DEV_WAIT_TIMEOUT);
            atomicExch(&sched[2], 1u);
            ok = false;
            break;
          }
          __nanosleep(256);
        }
        if (!ok) break;
      }
    }
    if (!__all_sync(FULL, ok)) break;
    __threadfence();  // the finished neighbours' positions are visible from here on

    // the group's frames, one cell after another, by the whole warp
    for (int g2 = 0; g2 < CPW; ++g2) {
      const int a2 = G * CPW + g2;
      if (a2 >= n_active) break;
      const int rep2 = act_rep[a2];
      const Geom& gg = rg[rep2];
      const SweepState* st2 = sts + rep2;
      const int col2 = st2->perm[ci];
      const int hx2 = gg.cells_x >> 1;
      const int la2 = a2 - gg.act_off;
      BuildArgs A;
      A.g = &gg;
      A.st = st2;
      A.cx = 2 * (la2 % hx2) + (col2 & 1);
      A.cy = 2 * (la2 / hx2) + (col2 >> 1);
      A.c = gg.cell_off + A.cy * gg.cells_x + A.cx;
      A.cap = cap;
      A.px = px;
      A.py = py;
      A.pid = pid;
      A.cnt = cnt;
      A.aux = aux;
      A.stage = hbase;
      A.rec = rec;
      A.a64 = a64;
      A.b64 = b64;
      A.lay = lay;
      A.gi = g2;
      A.err = err;
      build_frame<true, true>(A);
    }
    {
      int4* tz = reinterpret_cast<int4*>(tbase);
      const int4 z = make_int4(0, 0, 0, 0);
      for (int i = lane; i < (int)(fused_touch_bytes(lay) / 16); i += 32) tz[i] = z;
    }
    __syncwarp();

    __syncwarp();
    if constexpr (KIND == 1)
      run_group_iso<TPC, SCREEN>(f, hdr, hs.P, rg, sts, rep, a, valid, ci, px, py, cs, recs,
                                 rec_stride, err);
    else
      run_group<TPC, SCREEN, KIND == 2>(f, hs, hdr, rg, sts, rep, a, valid, ci, lay, px, py,
                                        cs, recs, rec_stride, replay, err);

    // publish: every lane's write-back is visible before the cell is marked
    __threadfence();
    __syncwarp();
    if (valid && sub == 0) {
      const int c = g.cell_off + cy * g.cells_x + cx;
      __threadfence();
      *(volatile unsigned*)&done[c] = epoch;
    }
    __syncwarp();
  }
}

size_t fused_smem_bytes(const RecLayout& lay, int fm) { return fused_warp_bytes(lay, fm); }
size_t fused_scratch_bytes(const RecLayout& lay) { return fused_fp64_bytes(lay); }

template <int TPC, int FM, int KIND>
static int configure_fused_t(size_t sm, int* blocks_per_sm) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return -1;
  int nb0 = 0, nb1 = 0;
  auto k0 = k_sweep_fused<TPC, false, FM, KIND>;
  auto k1 = k_sweep_fused<TPC, true, FM, KIND>;
  cudaFuncAttributes fa0, fa1;
  if (cudaFuncGetAttributes(&fa0, k0) != cudaSuccess ||
      cudaFuncGetAttributes(&fa1, k1) != cudaSuccess)
    return -1;
  const int mx0 = optin - (int)fa0.sharedSizeBytes, mx1 = optin - (int)fa1.sharedSizeBytes;
  if (sm > (size_t)mx0 || sm > (size_t)mx1) return -1;
  if (cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, mx0) != cudaSuccess ||
      cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, mx1) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb0, k0, 32, sm) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb1, k1, 32, sm) != cudaSuccess)
    return -1;
  *blocks_per_sm = nb0 < nb1 ? nb0 : nb1;
  return *blocks_per_sm > 0 ? 0 : -1;
}

int configure_fused(const RecLayout& lay, int tpc, int fm, int kind, int* blocks_per_sm) {
  const size_t sm = fused_smem_bytes(lay, fm);
#define ECMC_FCFG(T)                                                             \
  case T:                                                                        \
    return kind == 1   ? configure_fused_t<T, 0, 1>(sm, blocks_per_sm)           \
           : kind == 2 ? configure_fused_t<T, 0, 2>(sm, blocks_per_sm)           \
           : (fm == 1 ? configure_fused_t<T, 1, 0>(sm, blocks_per_sm)            \
                      : configure_fused_t<T, 0, 0>(sm, blocks_per_sm));
  switch (tpc) {
    ECMC_FCFG(1)
    ECMC_FCFG(2)
    ECMC_FCFG(4)
    ECMC_FCFG(8)
    ECMC_FCFG(16)
    ECMC_FCFG(32)
    default: return -1;
  }
#undef ECMC_FCFG
}

template <int TPC, bool SCREEN, int FM, int KIND = 0>
static int launch_fused_t(const DevBufs& b, const RecLayout& lay, int blocks, int records_on,
                          cudaStream_t s) {
  k_sweep_fused<TPC, SCREEN, FM, KIND><<<blocks, 32, fused_smem_bytes(lay, FM), s>>>(
      b.rg, b.state, b.act_rep, b.A_total, b.cap, b.px[b.cur], b.py[b.cur], b.pid[b.cur],
      b.count[b.cur], lay, b.cell_stats, records_on ? b.chain_recs : nullptr, b.rec_stride,
      b.replay, b.sched, b.done, b.wait_ns, b.wait_test, b.records, b.err);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_fused(const DevBufs& b, const RecLayout& lay, int tpc, int blocks, int records_on,
                 int precision, cudaStream_t s) {
  const bool scr = precision == 1;
#define ECMC_FCASE(T)                                                                      \
  case T:                                                                                  \
    if (b.iso)                                                                             \
      return scr ? launch_fused_t<T, true, 0, 1>(b, lay, blocks, records_on, s)            \
                 : launch_fused_t<T, false, 0, 1>(b, lay, blocks, records_on, s);          \
    if (b.reject)                                                                          \
      return scr ? launch_fused_t<T, true, 0, 2>(b, lay, blocks, records_on, s)            \
                 : launch_fused_t<T, false, 0, 2>(b, lay, blocks, records_on, s);          \
    return scr ? (b.fmode == 1 ? launch_fused_t<T, true, 1>(b, lay, blocks, records_on, s)    \
                               : launch_fused_t<T, true, 0>(b, lay, blocks, records_on, s))   \
               : (b.fmode == 1 ? launch_fused_t<T, false, 1>(b, lay, blocks, records_on, s)   \
                               : launch_fused_t<T, false, 0>(b, lay, blocks, records_on, s));
  switch (tpc) {
    ECMC_FCASE(1)
    ECMC_FCASE(2)
    ECMC_FCASE(4)
    ECMC_FCASE(8)
    ECMC_FCASE(16)
    ECMC_FCASE(32)
    default:
      return -1;
  }
#undef ECMC_FCASE
}

}  // namespace ecmc
