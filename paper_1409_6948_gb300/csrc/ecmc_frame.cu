// ecmc_frame.cu -- stage one colour's active cells into frame records
// (Sec. 3.4 step 6; the builder itself is in ecmc_build.cuh).  One block per
// active cell; the record is written to global memory for k_phase.
#include "ecmc_build.cuh"

namespace ecmc {

__global__ void __launch_bounds__(1024) k_frame_build(const Geom* __restrict__ rg, const SweepState* __restrict__ sts,
                              const int* __restrict__ act_rep, int cap, int colour_index,
                              const double* __restrict__ px, const double* __restrict__ py,
                              const int* __restrict__ pid, const int* __restrict__ cnt,
                              unsigned char* __restrict__ records, RecLayout lay,
                              unsigned char* __restrict__ stage, size_t stage_bytes, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int a = blockIdx.x;  // global active cell
  const int rep = act_rep[a];
  const Geom& g = rg[rep];
  const SweepState* st = sts + rep;
  const int colour = st->perm[colour_index];
  const int hx = g.cells_x >> 1;
  const int la = a - g.act_off;
  BuildArgs A;
  A.g = &g;
  A.st = st;
  A.cx = 2 * (la % hx) + (colour & 1);
  A.cy = 2 * (la / hx) + (colour >> 1);
  A.c = g.cell_off + A.cy * g.cells_x + A.cx;
  A.cap = cap;
  A.px = px;
  A.py = py;
  A.pid = pid;
  A.cnt = cnt;
  A.aux = smem;
  // staging area: shared memory, or a global region per block when the
  // frame is too large for shared memory
  A.stage = stage ? stage + (size_t)blockIdx.x * stage_bytes : smem + build_aux_bytes(blockDim.x);
  const int G = a / lay.cpw;
  A.rec = records + (size_t)G * lay.bytes;
  A.a64 = (double*)(A.rec + lay.off_a64);
  A.b64 = (double*)(A.rec + lay.off_b64);
  A.lay = lay;
  A.gi = a - G * lay.cpw;
  A.err = err;
  build_frame<false, false>(A);
}

// the staging area of one cell (shared memory, or global memory per block)
static size_t build_stage(const RecLayout& lay) { return build_stage_bytes(lay); }

static int build_threads(const RecLayout& lay) {
  int bt = 32;
  if (lay.cap_obj > 256) bt = 128;
  if (lay.cap_obj > 1024) bt = 256;
  if (lay.cap_obj > 4096) bt = 1024;
  return bt;
}

static size_t build_smem(const RecLayout& lay) {
  return build_aux_bytes(build_threads(lay)) + build_stage(lay);
}

void launch_frame_build(const DevBufs& b, const RecLayout& lay, int colour_index,
                        cudaStream_t s) {
  const int bt = build_threads(lay);
  const size_t sm = b.stage ? build_aux_bytes(bt) : build_smem(lay);
  k_frame_build<<<b.A_total, bt, sm, s>>>(b.rg, b.state, b.act_rep, b.cap, colour_index,
                                          b.px[b.cur], b.py[b.cur], b.pid[b.cur], b.count[b.cur],
                                          b.records, lay, b.stage, b.stage_bytes, b.err);
}

size_t frame_build_smem(const RecLayout& lay) { return build_smem(lay); }

size_t frame_stage_bytes(const RecLayout& lay) { return build_stage(lay); }

// largest amount the kernel can have, for the same reason as configure_phase
int configure_frame_build(const RecLayout& lay) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_frame_build) != cudaSuccess)
    return -1;
  const int mx = optin - (int)fa.sharedSizeBytes;
  if (build_smem(lay) > (size_t)mx) return -1;
  return cudaFuncSetAttribute(k_frame_build, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) ==
                 cudaSuccess
             ? 0
             : -1;
}

}  // namespace ecmc
