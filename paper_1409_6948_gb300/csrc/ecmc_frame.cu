// ecmc_frame.cu -- stage one colour's active cells into frame records.
//
// Sec. 3.4 step 6: while a cell is worked on, every disk outside it is
// frozen.  A chain of that cell can touch its members and every disk whose
// centre lies within sigma of the cell rectangle, including periodic images
// (with two cells per side the left and right neighbour are the same cell,
// and one disk may appear twice).  The builder places all of them in the
// cell's own frame -- the cell is [0,w] x [0,h] -- and sorts them into strips
// across the chain axis, so that the chain kernel only scans the strip of
// width 2 sigma around the moving disk (chains move along one axis, so the
// coordinate across the axis of every disk stays fixed during a sweep).
//
// One block per active cell.  The record is written in the interleaved
// layout of the chain kernel's groups ([index][cells per group]).
#include "ecmc_device.cuh"
#include "ecmc_internal.cuh"

namespace ecmc {

// Head of the builder's dynamic shared memory: neighbour cells and their
// prefix sums, then one 64-entry compaction buffer per warp.
constexpr size_t kBuildAuxHead = 128;
__host__ __device__ constexpr size_t build_aux_bytes(int threads) {
  return kBuildAuxHead + (size_t)(threads / 32) * 64 * sizeof(int2);
}

struct BuildSmem {
  double* a64;
  double* b64;
  int* key;
  int* slot;
  int* bin;
  int* fin;
  int* mrank;
  int* hist;
};

__global__ void k_frame_build(const Geom* __restrict__ rg, const SweepState* __restrict__ sts,
                              const int* __restrict__ act_rep, int cap, int colour_index,
                              const double* __restrict__ px, const double* __restrict__ py,
                              const int* __restrict__ pid, const int* __restrict__ cnt,
                              unsigned char* __restrict__ records, RecLayout lay,
                              unsigned char* __restrict__ stage, size_t stage_bytes, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_nobj, s_overflow, s_nnb;
  const int tid = threadIdx.x, bt = blockDim.x;
  const int a = blockIdx.x;  // global active cell
  const int rep = act_rep[a];
  const Geom& g = rg[rep];
  const SweepState* st = sts + rep;
  const int colour = st->perm[colour_index];
  const int hx = g.cells_x >> 1;
  const int la = a - g.act_off;
  const int cx = 2 * (la % hx) + (colour & 1);
  const int cy = 2 * (la / hx) + (colour >> 1);
  const int c = g.cell_off + cy * g.cells_x + cx;
  const int axis = st->axis;
  const double L = g.L, sigma = g.sigma;
  const double ox = st->sx + (double)cx * g.w;
  const double oy = st->sy + (double)cy * g.h;
  const double wl = g.w + sigma, hl = g.h + sigma;

  // shared-memory part that never moves to global memory: the neighbour
  // list and one compaction buffer of 64 entries per warp
  const int lane = tid & 31, warp = tid >> 5;
  int* s_nb = (int*)smem;      // distinct neighbour cells (<= 8)
  int* s_pre = s_nb + 8;       // prefix sums of their disk counts (<= 9)
  int2* wbuf = (int2*)(smem + kBuildAuxHead) + warp * 64;

  BuildSmem s;
  {
    // staging area: shared memory, or a global region per block when the
    // frame is too large for shared memory
    unsigned char* p = stage ? stage + (size_t)blockIdx.x * stage_bytes
                             : smem + build_aux_bytes(bt);
    s.a64 = (double*)p; p += sizeof(double) * lay.cap_obj;
    s.b64 = (double*)p; p += sizeof(double) * lay.cap_obj;
    s.key = (int*)p; p += sizeof(int) * lay.cap_obj;
    s.slot = (int*)p; p += sizeof(int) * lay.cap_obj;
    s.bin = (int*)p; p += sizeof(int) * lay.cap_obj;
    s.fin = (int*)p; p += sizeof(int) * lay.cap_obj;
    s.mrank = (int*)p; p += sizeof(int) * lay.cap_mem;
    s.hist = (int*)p; p += sizeof(int) * (lay.nbin + 1);
  }
  if (tid == 0) {
    s_nobj = 0;
    s_overflow = 0;
    // distinct neighbour cells of the 3x3 block; their disks are visited as
    // one index range [0, s_pre[nnb])
    int nnb = 0;
    for (int oyc = -1; oyc <= 1; ++oyc)
      for (int oxc = -1; oxc <= 1; ++oxc) {
        const int qx = ((cx + oxc) % g.cells_x + g.cells_x) % g.cells_x;
        const int qy = ((cy + oyc) % g.cells_y + g.cells_y) % g.cells_y;
        const int q = g.cell_off + qy * g.cells_x + qx;
        if (q == c) continue;
        bool dup = false;
        for (int e = 0; e < nnb; ++e) dup |= (s_nb[e] == q);
        if (!dup) s_nb[nnb++] = q;
      }
    int run = 0;
    for (int e = 0; e < nnb; ++e) {
      s_pre[e] = run;
      run += min(cnt[s_nb[e]], cap);
    }
    for (int e = nnb; e <= 8; ++e) s_pre[e] = run;
    s_nnb = nnb;
  }
  __syncthreads();

  // members, in the cell frame
  const double hL = 0.5 * L;
  const int nc = min(cnt[c], cap);
  for (int k = tid; k < nc; k += bt) {
    const int64_t q = (int64_t)c * cap + k;
    const double X = wrap_half_i(px[q] - ox, L, hL);
    const double Y = wrap_half_i(py[q] - oy, L, hL);
    const int i = atomicAdd(&s_nobj, 1);
    s.a64[i] = axis == 0 ? X : Y;
    s.b64[i] = axis == 0 ? Y : X;
    s.key[i] = pid[q] * 16 + 4;
    s.slot[i] = (int)q;
  }
  __syncthreads();
  // every thread takes the member count before any thread appends a frozen
  // image (blocks of several warps would otherwise race)
  const int nmem = s_nobj;
  __syncthreads();

  // frozen images within sigma of the cell rectangle.  An FP32 screen with a
  // margin well above its rounding error (|error| < 4 * 2^-23 L) discards the
  // disks that no image can bring near the cell; the others take the FP64
  // test, so the frame is exactly the one the FP64 test alone would build.
  // The survivors of the screen are compacted per warp before the FP64 work,
  // so that every FP64 instruction serves 32 candidates (an FP64 warp
  // instruction costs the same whatever the number of active lanes).
  const float Lf = (float)L;
  const float oxf = to_float_trunc(ox), oyf = to_float_trunc(oy);
  const float mf = 8.0f * 1.1920929e-7f * Lf + 1e-6f;
  const float xlo = -(float)sigma - mf, xhi = (float)wl + mf;
  const float ylo = -(float)sigma - mf, yhi = (float)hl + mf;
  const int nnb = s_nnb, T = s_pre[nnb];
  const unsigned FULL = 0xffffffffu;

  // FP64 placement of one screened disk: the wrapped difference, then the
  // images the screen kept (offsets j*L of the unwrapped difference; an FP64
  // image k of the wrapped difference is offset j = k - (wrap shift))
  auto place = [&](int2 v) {
    // neighbour e (3 bits) and bucket slot k (29 bits), packed unsigned
    const unsigned ek = (unsigned)v.x;
    const int e = (int)(ek >> 29), k = (int)(ek & ((1u << 29) - 1u));
    const unsigned imgx = (unsigned)v.y & 31u, imgy = (unsigned)v.y >> 5;
    const int64_t q = (int64_t)s_nb[e] * cap + k;
    const double rx = px[q] - ox, ry = py[q] - oy;
    const int swx = !dlt(rx, hL) ? 1 : (dlt(rx, -hL) ? -1 : 0);
    const int swy = !dlt(ry, hL) ? 1 : (dlt(ry, -hL) ? -1 : 0);
    // wrap_half(r, L): r - L, r + L (as r - (-L)) or r - 0
    const double X0 = rx - (swx == 0 ? 0.0 : flip_if(L, swx < 0));
    const double Y0 = ry - (swy == 0 ? 0.0 : flip_if(L, swy < 0));
    const int id = pid[q];
    for (int kx = -1; kx <= 1; ++kx) {
      if (!(imgx & (1u << (kx - swx + 2)))) continue;
      const double X = (kx == 0) ? X0 : X0 + flip_if(L, kx < 0);
      if (!(dlt(-sigma, X) && dlt(X, wl))) continue;
      for (int ky = -1; ky <= 1; ++ky) {
        if (!(imgy & (1u << (ky - swy + 2)))) continue;
        const double Y = (ky == 0) ? Y0 : Y0 + flip_if(L, ky < 0);
        if (!(dlt(-sigma, Y) && dlt(Y, hl))) continue;
        const int i = atomicAdd(&s_nobj, 1);
        if (i >= lay.cap_obj) {
          s_overflow = 1;
          continue;
        }
        s.a64[i] = axis == 0 ? X : Y;
        s.b64[i] = axis == 0 ? Y : X;
        s.key[i] = id * 16 + (kx + 1) * 3 + (ky + 1);
        s.slot[i] = -1;
      }
    }
  };

  int nbuf = 0;  // warp-uniform fill of this warp's buffer (< 32 between chunks)
  for (int base = warp * 32; base < T; base += bt) {
    const int idx = base + lane;
    bool keep = false;
    int2 ent = make_int2(0, 0);
    if (idx < T) {
      int e = 0;
      while (e + 1 < nnb && s_pre[e + 1] <= idx) ++e;
      const int k = idx - s_pre[e];
      const int64_t q = (int64_t)s_nb[e] * cap + k;
      const float rxf = to_float_trunc(px[q]) - oxf, ryf = to_float_trunc(py[q]) - oyf;
      unsigned imgx = 0, imgy = 0;
      for (int j = -2; j <= 2; ++j) {
        const float Xf = rxf + (float)j * Lf, Yf = ryf + (float)j * Lf;
        imgx |= (Xf > xlo && Xf < xhi) ? (1u << (j + 2)) : 0u;
        imgy |= (Yf > ylo && Yf < yhi) ? (1u << (j + 2)) : 0u;
      }
      keep = imgx && imgy;
      ent = make_int2((int)(((unsigned)e << 29) | (unsigned)k), (int)(imgx | (imgy << 5)));
    }
    const unsigned bal = __ballot_sync(FULL, keep);
    if (keep) wbuf[nbuf + __popc(bal & ((1u << lane) - 1u))] = ent;
    nbuf += __popc(bal);
    __syncwarp();
    if (nbuf >= 32) {
      const int2 v = wbuf[lane];
      __syncwarp();
      if (lane < nbuf - 32) wbuf[lane] = wbuf[lane + 32];
      nbuf -= 32;
      __syncwarp();
      place(v);
    }
  }
  if (lane < nbuf) place(wbuf[lane]);
  for (int k = tid; k <= lay.nbin; k += bt) s.hist[k] = 0;
  __syncthreads();
  if (s_overflow) {
    if (tid == 0) atomicCAS(err, DEV_OK, DEV_CAPACITY);
  }
  const int nobj = min(s_nobj, lay.cap_obj);

  // members ranked by disk id (start disks are drawn by rank)
  for (int i = tid; i < nmem; i += bt) {
    const int ki = s.key[i];
    int r = 0;
    for (int k = 0; k < nmem; ++k) r += (s.key[k] < ki);
    s.mrank[r] = i;
  }
  // strips across the chain axis: bin of the FP32 coordinate
  for (int i = tid; i < nobj; i += bt) {
    const float b32 = to_float_trunc(s.b64[i]);
    int kb = (int)((b32 + g.sigf) * g.inv_bin_w);
    kb = kb < 0 ? 0 : (kb >= lay.nbin ? lay.nbin - 1 : kb);
    s.bin[i] = kb;
    atomicAdd(&s.hist[kb], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int k = 0; k < lay.nbin; ++k) {
      const int v = s.hist[k];
      s.hist[k] = run;
      run += v;
    }
    s.hist[lay.nbin] = run;
  }
  __syncthreads();

  // write the record of group G, column gi
  const int cpw = lay.cpw;
  const int G = a / cpw, gi = a - G * cpw;
  unsigned char* rec = records + (size_t)G * lay.bytes;
  int* hdr = (int*)(rec + lay.off_hdr);
  int* bst = (int*)(rec + lay.off_bstart);
  int* mr = (int*)(rec + lay.off_mrank);
  int* ms = (int*)(rec + lay.off_mslot);
  float* a32 = (float*)(rec + lay.off_a32);
  float* b32 = (float*)(rec + lay.off_b32);
  double* a64 = (double*)(rec + lay.off_a64);
  double* b64 = (double*)(rec + lay.off_b64);
  int* key = (int*)(rec + lay.off_key);
  int* info = (int*)(rec + lay.off_info);
  if (tid == 0) {
    hdr[gi] = nobj;
    hdr[cpw + gi] = nmem;
  }
  for (int k = tid; k <= lay.nbin; k += bt) bst[k * cpw + gi] = s.hist[k];
  __syncthreads();
  for (int i = tid; i < nobj; i += bt) {
    const int f = atomicAdd(&s.hist[s.bin[i]], 1);
    s.fin[i] = f;
    a32[f * cpw + gi] = to_float_trunc(s.a64[i]);
    b32[f * cpw + gi] = to_float_trunc(s.b64[i]);
    a64[f * cpw + gi] = s.a64[i];
    b64[f * cpw + gi] = s.b64[i];
    key[f * cpw + gi] = s.key[i];
    info[f * cpw + gi] = -1;
  }
  __syncthreads();
  for (int r = tid; r < nmem; r += bt) {
    const int i = s.mrank[r];
    mr[r * cpw + gi] = s.fin[i];
    ms[r * cpw + gi] = s.slot[i];
    info[s.fin[i] * cpw + gi] = r;
  }
}

// the staging area of one cell (shared memory, or global memory per block)
static size_t build_stage(const RecLayout& lay) {
  return align16((sizeof(double) * 2 + sizeof(int) * 4) * (size_t)lay.cap_obj +
                 sizeof(int) * (size_t)lay.cap_mem + sizeof(int) * (size_t)(lay.nbin + 1) + 64);
}

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
