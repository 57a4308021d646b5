// ecmc_build.cuh -- building one cell's frame record (Sec. 3.4 step 6).
//
// While a cell is worked on, every disk outside it is frozen.  A chain of
// that cell can touch its members and every disk whose centre lies within
// sigma of the cell rectangle, including periodic images (with two cells per
// side the left and right neighbour are the same cell, and one disk may
// appear twice).  The builder places all of them in the cell's own frame --
// the cell is [0,w] x [0,h] -- and sorts them into strips across the chain
// axis, so that the chain kernel only scans the strip of width 2 sigma around
// the moving disk (chains move along one axis, so the coordinate across the
// axis of every disk stays fixed during a sweep).  The record is written in
// the interleaved layout of the chain kernel's groups ([index][cells per
// group]).
//
// Two users: k_frame_build (one block per active cell, WARP = false) and the
// persistent sweep kernel (one warp builds the frames of its group one after
// another into shared memory, WARP = true).  In the persistent kernel other
// warps move disks while this one reads positions, so positions are read
// through L2 only (CG = true): a line cached in L1 by an earlier item could
// be stale.
#pragma once

#include "ecmc_device.cuh"
#include "ecmc_internal.cuh"

namespace ecmc {

// Head of a builder's shared scratch: its scalars, the neighbour cells and
// their prefix sums; then one 64-entry compaction buffer per warp.
constexpr size_t kBuildAuxHead = 128;
__host__ __device__ constexpr size_t build_aux_bytes(int threads) {
  return kBuildAuxHead + (size_t)(threads / 32) * 64 * sizeof(int2);
}

// Staging area of one cell: objects before they are sorted into strips.
__host__ __device__ inline size_t build_stage_bytes(const RecLayout& lay) {
  return align16((sizeof(double) * 2 + sizeof(int) * 4) * (size_t)lay.cap_obj +
                 sizeof(int) * (size_t)lay.cap_mem + sizeof(int) * (size_t)(lay.nbin + 1) + 64);
}

struct BuildArgs {
  const Geom* g;
  const SweepState* st;
  int cx, cy, c;              // cell in the replica's grid, global cell
  int cap;                    // bucket capacity
  const double* px;           // bucketed positions
  const double* py;
  const int* pid;
  const int* cnt;
  unsigned char* aux;         // build_aux_bytes(threads) of shared memory
  unsigned char* stage;       // build_stage_bytes(lay), shared or global memory
  unsigned char* rec;         // record of the group: header, strips, members, FP32 part
  double* a64;                // the group's FP64 coordinates along / across the axis
  double* b64;                // (in the record, or in a separate scratch area)
  RecLayout lay;
  int gi;                     // column of this cell in the record
  int* err;
};

template <bool CG>
__device__ __forceinline__ double load_pos(const double* p) {
  return CG ? __ldcg(p) : *p;
}

// Build the frame of one cell.  WARP: the calling warp alone (tid = lane,
// 32 threads, __syncwarp); else the whole block.
template <bool WARP, bool CG>
__device__ void build_frame(const BuildArgs& A) {
  const int tid = WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
  const int bt = WARP ? 32 : (int)blockDim.x;
  auto sync = [] {
    if (WARP) __syncwarp();
    else __syncthreads();
  };
  const Geom& g = *A.g;
  const SweepState* st = A.st;
  const RecLayout& lay = A.lay;
  const int cx = A.cx, cy = A.cy, c = A.c, cap = A.cap;
  const int axis = st->axis;
  const double L = g.L, sigma = g.sigma;
  const double ox = st->sx + (double)cx * g.w;
  const double oy = st->sy + (double)cy * g.h;
  const double wl = g.w + sigma, hl = g.h + sigma;
  const unsigned FULL = 0xffffffffu;

  int* s_scal = (int*)A.aux;  // [0] objects, [1] overflow, [2] neighbour cells
  int* s_nb = s_scal + 4;     // distinct neighbour cells (<= 8)
  int* s_pre = s_nb + 8;      // prefix sums of their disk counts (<= 9)
  const int lane = tid & 31, warp = tid >> 5;
  int2* wbuf = (int2*)(A.aux + kBuildAuxHead) + warp * 64;

  double* s_a64;
  double* s_b64;
  int *s_key, *s_slot, *s_bin, *s_fin, *s_mrank, *s_hist;
  {
    unsigned char* p = A.stage;
    s_a64 = (double*)p; p += sizeof(double) * lay.cap_obj;
    s_b64 = (double*)p; p += sizeof(double) * lay.cap_obj;
    s_key = (int*)p; p += sizeof(int) * lay.cap_obj;
    s_slot = (int*)p; p += sizeof(int) * lay.cap_obj;
    s_bin = (int*)p; p += sizeof(int) * lay.cap_obj;
    s_fin = (int*)p; p += sizeof(int) * lay.cap_obj;
    s_mrank = (int*)p; p += sizeof(int) * lay.cap_mem;
    s_hist = (int*)p;
  }

  if (tid < 32) {
    // distinct neighbour cells of the 3x3 block, one per lane (with two
    // cells per side the left and right neighbour coincide), and the prefix
    // sums of their disk counts: their disks are visited as one index range
    int q = -1;
    if (tid < 9) {
      int qx = cx + tid % 3 - 1, qy = cy + tid / 3 - 1;
      qx += qx < 0 ? g.cells_x : 0;
      qx -= qx >= g.cells_x ? g.cells_x : 0;
      qy += qy < 0 ? g.cells_y : 0;
      qy -= qy >= g.cells_y ? g.cells_y : 0;
      q = g.cell_off + qy * g.cells_x + qx;
      if (q == c) q = -1;
    }
    const unsigned lower = (1u << tid) - 1u;
    const unsigned same = __match_any_sync(FULL, q);
    const bool keep = q >= 0 && (same & lower) == 0;
    const unsigned kept = __ballot_sync(FULL, keep);
    const int nq = keep ? min(A.cnt[q], cap) : 0;
    int incl = nq;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, o);
      if (tid >= o) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    const int nnb = __popc(kept);
    if (keep) {
      const int pos = __popc(kept & lower);
      s_nb[pos] = q;
      s_pre[pos] = incl - nq;
    }
    if (tid >= nnb && tid <= 8) s_pre[tid] = total;
    if (tid == 0) {
      s_scal[0] = 0;
      s_scal[1] = 0;
      s_scal[2] = nnb;
    }
  }
  sync();

  // members, in the cell frame
  const double hL = 0.5 * L;
  const int nc = min(A.cnt[c], cap);
  for (int k = tid; k < nc; k += bt) {
    const int64_t q = (int64_t)c * cap + k;
    const double X = wrap_half_i(load_pos<CG>(A.px + q) - ox, L, hL);
    const double Y = wrap_half_i(load_pos<CG>(A.py + q) - oy, L, hL);
    const int i = atomicAdd(&s_scal[0], 1);
    s_a64[i] = axis == 0 ? X : Y;
    s_b64[i] = axis == 0 ? Y : X;
    s_key[i] = A.pid[q] * 16 + 4;
    s_slot[i] = (int)q;
  }
  sync();
  // every thread takes the member count before any thread appends a frozen
  // image (blocks of several warps would otherwise race)
  const int nmem = s_scal[0];
  sync();

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
  const int nnb = s_scal[2], T = s_pre[nnb];

  // FP64 placement of one screened disk: the wrapped difference, then the
  // images the screen kept (offsets j*L of the unwrapped difference; an FP64
  // image k of the wrapped difference is offset j = k - (wrap shift))
  auto place = [&](int2 v) {
    // neighbour e (3 bits) and bucket slot k (29 bits), packed unsigned
    const unsigned ek = (unsigned)v.x;
    const int e = (int)(ek >> 29), k = (int)(ek & ((1u << 29) - 1u));
    const unsigned imgx = (unsigned)v.y & 31u, imgy = (unsigned)v.y >> 5;
    const int64_t q = (int64_t)s_nb[e] * cap + k;
    const double rx = load_pos<CG>(A.px + q) - ox, ry = load_pos<CG>(A.py + q) - oy;
    const int swx = !dlt(rx, hL) ? 1 : (dlt(rx, -hL) ? -1 : 0);
    const int swy = !dlt(ry, hL) ? 1 : (dlt(ry, -hL) ? -1 : 0);
    // wrap_half(r, L): r - L, r + L (as r - (-L)) or r - 0
    const double X0 = rx - (swx == 0 ? 0.0 : flip_if(L, swx < 0));
    const double Y0 = ry - (swy == 0 ? 0.0 : flip_if(L, swy < 0));
    const int id = A.pid[q];
    for (int kx = -1; kx <= 1; ++kx) {
      if (!(imgx & (1u << (kx - swx + 2)))) continue;
      const double X = (kx == 0) ? X0 : X0 + flip_if(L, kx < 0);
      if (!(dlt(-sigma, X) && dlt(X, wl))) continue;
      for (int ky = -1; ky <= 1; ++ky) {
        if (!(imgy & (1u << (ky - swy + 2)))) continue;
        const double Y = (ky == 0) ? Y0 : Y0 + flip_if(L, ky < 0);
        if (!(dlt(-sigma, Y) && dlt(Y, hl))) continue;
        const int i = atomicAdd(&s_scal[0], 1);
        if (i >= lay.cap_obj) {
          s_scal[1] = 1;
          continue;
        }
        s_a64[i] = axis == 0 ? X : Y;
        s_b64[i] = axis == 0 ? Y : X;
        s_key[i] = id * 16 + (kx + 1) * 3 + (ky + 1);
        s_slot[i] = -1;
      }
    }
  };

  // The offsets r = x - o lie in (-L, L) (x in [0, L), the frame origin o in
  // [0, L)), and the frame (-sigma, w + sigma) is shorter than L, so only the
  // images r - L, r, r + L can fall in it: bits 1, 2, 3 of the image masks.
  // The neighbour of disk idx is searched from the previous round's (idx
  // only grows).
  int nbuf = 0;  // warp-uniform fill of this warp's buffer (< 32 between chunks)
  int e_run = 0;
  // one call site of place() (the final partial buffer is flushed in the
  // pass after the last chunk), so that its code is emitted once
  for (int base = warp * 32;; base += bt) {
    const bool more = base < T;  // warp-uniform
    if (more) {
      const int idx = base + lane;
      bool keep = false;
      int2 ent = make_int2(0, 0);
      if (idx < T) {
        int e = e_run;
        while (e + 1 < nnb && s_pre[e + 1] <= idx) ++e;
        e_run = e;
        const int k = idx - s_pre[e];
        const int64_t q = (int64_t)s_nb[e] * cap + k;
        const float rxf = to_float_trunc(load_pos<CG>(A.px + q)) - oxf;
        const float ryf = to_float_trunc(load_pos<CG>(A.py + q)) - oyf;
        unsigned imgx = 0, imgy = 0;
        for (int j = -1; j <= 1; ++j) {
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
    }
    if (nbuf >= 32 || (!more && nbuf > 0)) {
      const int2 v = wbuf[lane];
      const bool has = lane < nbuf;
      __syncwarp();
      if (lane < nbuf - 32) wbuf[lane] = wbuf[lane + 32];
      nbuf = nbuf > 32 ? nbuf - 32 : 0;
      __syncwarp();
      if (has) place(v);
    }
    if (!more) break;
  }
  for (int k = tid; k <= lay.nbin; k += bt) s_hist[k] = 0;
  sync();
  if (s_scal[1]) {
    if (tid == 0) atomicCAS(A.err, DEV_OK, DEV_CAPACITY);
  }
  const int nobj = min(s_scal[0], lay.cap_obj);

  // members ranked by disk id (start disks are drawn by rank)
  for (int i = tid; i < nmem; i += bt) {
    const int ki = s_key[i];
    int r = 0;
    for (int k = 0; k < nmem; ++k) r += (s_key[k] < ki);
    s_mrank[r] = i;
  }
  // strips across the chain axis: bin of the FP32 coordinate
  for (int i = tid; i < nobj; i += bt) {
    const float b32 = to_float_trunc(s_b64[i]);
    int kb = (int)((b32 + g.sigf) * g.inv_bin_w);
    kb = kb < 0 ? 0 : (kb >= lay.nbin ? lay.nbin - 1 : kb);
    s_bin[i] = kb;
    atomicAdd(&s_hist[kb], 1);
  }
  sync();
  if (tid < 32) {
    // exclusive prefix sums of the strip counts, 32 strips at a time
    int carry = 0;
    for (int k0 = 0; k0 < lay.nbin; k0 += 32) {
      const int k = k0 + tid;
      const int v = k < lay.nbin ? s_hist[k] : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, incl, o);
        if (tid >= o) incl += u;
      }
      if (k < lay.nbin) s_hist[k] = carry + incl - v;
      carry += __shfl_sync(FULL, incl, 31);
    }
    if (tid == 0) s_hist[lay.nbin] = carry;
  }
  sync();

  // write the record, column gi
  const int cpw = lay.cpw, gi = A.gi;
  unsigned char* rec = A.rec;
  int* hdr = (int*)(rec + lay.off_hdr);
  int* bst = (int*)(rec + lay.off_bstart);
  int* mr = (int*)(rec + lay.off_mrank);
  int* ms = (int*)(rec + lay.off_mslot);
  float* a32 = (float*)(rec + lay.off_a32);
  float* b32 = (float*)(rec + lay.off_b32);
  double* a64 = A.a64;
  double* b64 = A.b64;
  int* key = (int*)(rec + lay.off_key);
  int* info = (int*)(rec + lay.off_info);
  if (tid == 0) {
    hdr[gi] = nobj;
    hdr[cpw + gi] = nmem;
  }
  for (int k = tid; k <= lay.nbin; k += bt) bst[k * cpw + gi] = s_hist[k];
  sync();
  for (int i = tid; i < nobj; i += bt) {
    const int f = atomicAdd(&s_hist[s_bin[i]], 1);
    s_fin[i] = f;
    a32[f * cpw + gi] = to_float_trunc(s_a64[i]);
    b32[f * cpw + gi] = to_float_trunc(s_b64[i]);
    a64[f * cpw + gi] = s_a64[i];
    b64[f * cpw + gi] = s_b64[i];
    key[f * cpw + gi] = s_key[i];
    info[f * cpw + gi] = -1;
  }
  sync();
  for (int r = tid; r < nmem; r += bt) {
    const int i = s_mrank[r];
    mr[r * cpw + gi] = s_fin[i];
    ms[r * cpw + gi] = s_slot[i];
    info[s_fin[i] * cpw + gi] = r;
  }
  sync();
}

}  // namespace ecmc
