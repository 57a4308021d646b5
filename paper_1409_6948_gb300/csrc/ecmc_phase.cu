// ecmc_phase.cu -- the chain kernel: one colour phase of the sweep, one
// launch per phase, frames staged by k_frame_build (the chain loop itself is
// in ecmc_chain.cuh).
#include "ecmc_chain.cuh"
#include "ecmc_chain_iso.cuh"

namespace ecmc {

// FMODE 0: the warp copies its group's whole record into shared memory;
// FMODE 1: only the light part (FP32 coordinates, keys, strips, members), the
// FP64 coordinates are read and written in place in global memory (more
// cells fit in shared memory at once); FMODE 2: the whole record is used in
// place in global memory (cells too large for shared memory).
template <int TPC, bool SCREEN, int FMODE, int KIND = 0>
__global__ void __launch_bounds__(256) k_phase(const Geom* __restrict__ rg,
                                               const SweepState* __restrict__ sts,
                                               const int* __restrict__ act_rep, int colour_index,
                                               unsigned char* __restrict__ records,
                                               unsigned char* __restrict__ gtouch, RecLayout lay,
                                               int n_active, double* __restrict__ px,
                                               double* __restrict__ py, CellStats* __restrict__ cs,
                                               ChainRec* __restrict__ recs, int rec_stride,
                                               int replay, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int CPW = 32 / TPC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_groups = (n_active + CPW - 1) / CPW;
  const int G = blockIdx.x * (blockDim.x >> 5) + warp;
  if (G >= n_groups) return;

  const size_t rec_bytes = lay.bytes;
  const size_t t_bytes = align16((size_t)lay.cap_obj * CPW);
  const size_t h_bytes = kHistLegBytes * kHist * CPW;
  unsigned char* const grec = records + (size_t)G * rec_bytes;
  unsigned char* base;
  unsigned char* tbase;
  unsigned char* hbase;
  if (FMODE == 2) {
    base = grec;
    tbase = gtouch + (size_t)G * t_bytes;
    hbase = smem + (size_t)warp * h_bytes;
  } else {
    const size_t copy = FMODE == 1 ? lay.light_bytes : rec_bytes;
    base = smem + (size_t)warp * (copy + t_bytes + h_bytes);
    tbase = base + copy;
    hbase = tbase + t_bytes;
    const int4* src = reinterpret_cast<const int4*>(grec);
    int4* dst = reinterpret_cast<int4*>(base);
    const int n16 = (int)(copy / 16);
    for (int i = lane; i < n16; i += 32) dst[i] = src[i];
  }
  {
    int4* tz = reinterpret_cast<int4*>(tbase);
    const int4 z = make_int4(0, 0, 0, 0);
    for (int i = lane; i < (int)(t_bytes / 16); i += 32) tz[i] = z;
  }
  __syncwarp();

  Frame f;
  f.cpw = CPW;
  f.bst = (const int*)(base + lay.off_bstart);
  f.mrank = (const int*)(base + lay.off_mrank);
  f.mslot = (const int*)(base + lay.off_mslot);
  f.a32 = (float*)(base + lay.off_a32);
  f.b32 = (float*)(base + lay.off_b32);
  f.a64 = (double*)((FMODE == 1 ? grec : base) + lay.off_a64);
  f.b64 = (double*)((FMODE == 1 ? grec : base) + lay.off_b64);
  f.key = (const int*)(base + lay.off_key);
  f.info = (const int*)(base + lay.off_info);
  f.touched = tbase;
  const int* hdr = (const int*)(base + lay.off_hdr);
  LegHist hs;  // interleaved [leg][group] like the frame
  hs.P = (double*)hbase;
  hs.step = hs.P + kHist * CPW;
  hs.addb = hs.step + kHist * CPW;
  hs.m = (int*)(hs.addb + kHist * CPW);
  hs.flags = hs.m + kHist * CPW;

  const int gi = lane / TPC;
  const int a = G * CPW + gi;  // global active cell of this lane group
  const bool valid = a < n_active;
  const int rep = valid ? act_rep[a] : act_rep[n_active - 1];
  if constexpr (KIND == 1)
    run_group_iso<TPC, SCREEN>(f, hdr, hs.P, rg, sts, rep, a, valid, colour_index, px, py, cs,
                               recs, rec_stride, err);
  else
    run_group<TPC, SCREEN, KIND == 2>(f, hs, hdr, rg, sts, rep, a, valid, colour_index, lay, px,
                                      py, cs, recs, rec_stride, replay, err);
}

size_t phase_smem_bytes(const RecLayout& lay, int warps_per_block, int fmode) {
  const size_t hist = kHistLegBytes * kHist * (size_t)lay.cpw;
  if (fmode == 2) return (size_t)warps_per_block * hist;
  const size_t copy = fmode == 1 ? lay.light_bytes : lay.bytes;
  return (size_t)warps_per_block * (copy + align16((size_t)lay.cap_obj * lay.cpw) + hist);
}

template <int TPC, bool SCREEN>
static int launch_t(const DevBufs& b, const RecLayout& lay, int colour_index, int warps,
                    int records_on, cudaStream_t s) {
  const int n_active = b.A_total;
  const int cpw = 32 / TPC;
  const int n_groups = (n_active + cpw - 1) / cpw;
  const int blocks = (n_groups + warps - 1) / warps;
  const size_t sm = phase_smem_bytes(lay, warps, b.fmode);
#define ECMC_PHASE(FM, KIND)                                                               \
  k_phase<TPC, SCREEN, FM, KIND><<<blocks, 32 * warps, sm, s>>>(                           \
      b.rg, b.state, b.act_rep, colour_index, b.records, b.gtouch, lay, n_active,          \
      b.px[b.cur], b.py[b.cur], b.cell_stats, records_on ? b.chain_recs : nullptr,         \
      b.rec_stride, b.replay, b.err)
  const int kind = chain_kind(b);
  if (kind == 1) {
    if (b.fmode == 2) ECMC_PHASE(2, 1);
    else if (b.fmode == 1) ECMC_PHASE(1, 1);
    else ECMC_PHASE(0, 1);
  } else if (kind == 2) {
    if (b.fmode == 2) ECMC_PHASE(2, 2);
    else if (b.fmode == 1) ECMC_PHASE(1, 2);
    else ECMC_PHASE(0, 2);
  } else {
    if (b.fmode == 2) ECMC_PHASE(2, 0);
    else if (b.fmode == 1) ECMC_PHASE(1, 0);
    else ECMC_PHASE(0, 0);
  }
#undef ECMC_PHASE
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Largest dynamic shared memory a launch of `fn` may request: the device's
// opt-in per-block amount minus the kernel's static shared memory.
template <typename F>
static int max_dynamic_smem(F fn, int* out) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess ||
      cudaFuncGetAttributes(&fa, fn) != cudaSuccess)
    return -1;
  *out = optin - (int)fa.sharedSizeBytes;
  return 0;
}

template <typename F>
static int configure_fn(F fn, size_t need) {
  int mx = 0;
  if (max_dynamic_smem(fn, &mx) || need > (size_t)mx) return -1;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) == cudaSuccess
             ? 0
             : -1;
}

template <int TPC, int FM>
static int configure_t(size_t sm) {
  if (configure_fn(k_phase<TPC, true, FM>, sm)) return -1;
  if (configure_fn(k_phase<TPC, false, FM>, sm)) return -1;
  if (configure_fn(k_phase<TPC, false, FM, 1>, sm)) return -1;
  if (configure_fn(k_phase<TPC, true, FM, 1>, sm)) return -1;
  if (configure_fn(k_phase<TPC, false, FM, 2>, sm)) return -1;
  if (configure_fn(k_phase<TPC, true, FM, 2>, sm)) return -1;
  return 0;
}

// The attribute is a per-kernel, per-process maximum: request the largest
// amount the kernel can have, so that a handle with small frames never lowers
// the limit that a handle with larger frames needs.
int configure_phase(const RecLayout& lay, int tpc, int warps, int fmode) {
  const size_t sm = phase_smem_bytes(lay, warps, fmode);
#define ECMC_CFG(T)                                                          \
  case T:                                                                    \
    return fmode == 1 ? configure_t<T, 1>(sm) : configure_t<T, 0>(sm);
  if (fmode == 2) {
    // frames in global memory: only the leg histories use shared memory
    switch (tpc) {
      case 1: return configure_t<1, 2>(sm);
      case 2: return configure_t<2, 2>(sm);
      case 4: return configure_t<4, 2>(sm);
      case 8: return configure_t<8, 2>(sm);
      case 16: return configure_t<16, 2>(sm);
      case 32: return configure_t<32, 2>(sm);
      default: return -1;
    }
  }
  switch (tpc) {
    ECMC_CFG(1)
    ECMC_CFG(2)
    ECMC_CFG(4)
    ECMC_CFG(8)
    ECMC_CFG(16)
    ECMC_CFG(32)
    default: return -1;
  }
#undef ECMC_CFG
}

int launch_phase(const DevBufs& b, const RecLayout& lay, int colour_index, int tpc, int warps,
                 int records_on, int precision, cudaStream_t s) {
  const bool scr = precision == 1;
#define ECMC_CASE(T)                                                           \
  case T:                                                                      \
    return scr ? launch_t<T, true>(b, lay, colour_index, warps, records_on, s) \
               : launch_t<T, false>(b, lay, colour_index, warps, records_on, s);
  switch (tpc) {
    ECMC_CASE(1)
    ECMC_CASE(2)
    ECMC_CASE(4)
    ECMC_CASE(8)
    ECMC_CASE(16)
    ECMC_CASE(32)
    default:
      return -1;
  }
#undef ECMC_CASE
}

}  // namespace ecmc
