// Per-thread target tiles of the StepForward / StepBackward pair sums, and
// the TMA pipeline that streams a range of sources through shared memory.
// Both the split-partial kernels (pair_kernels.cu) and the fused step kernels
// (step_kernels.cu) are built from these pieces.
//
// Packed arithmetic.  Sources sit in memory as pair records: two landmarks
// interleaved per coordinate (layout in gs_internal.h; D float4 per record
// for landmarks in D = 3 or 2 dimensions).  The inner loop uses
// the sm_100+ paired FP32 instructions (__fadd2_rn, __fmul2_rn, __ffma2_rn).
// Each instruction applies one target to two sources, which halves the issue
// slots spent on FP32 work.  Positions are stored negated, so q_i - q_j is a
// single paired add.  The Gaussian is one MUFU ex2 per pair, on prescaled
// coordinates.
//
// A thread holds R targets in registers.  The threads of a CTA form one or
// more warp groups; each group holds the same targets (base + r*TG, r < R,
// TG threads per group) and takes its own share of every staged chunk of
// sources, so a CTA with W groups splits its sources W ways.  The whole warp
// reads the same source record, so the shared-memory load is a broadcast.
// Sums are plain FP32 over a sub-block of at most kSub sources, then the two
// halves of each paired accumulator are added and folded into a Kahan (sum,
// compensation) pair.
#pragma once

#include "gs_device.cuh"
#include "gs_internal.h"

namespace gs {

// Sources per plain-FP32 sub-block before a Kahan fold: one staged chunk.
// Measured on GB300 in whole gradients (T = 20), 128 against 64: -1.7 % at
// N = 4096 and 16384, both kernels.
constexpr int kSub = 128;
constexpr int kUnroll = 8;  // split lengths are multiples of this

// kStages chunk buffers for NA record arrays (kChunk sources = kChunk/2
// records of D float4 each, D the dimension of the landmarks).  The
// mbarriers live outside (struct Pipe), so this memory can be reused once
// the last chunk has been consumed.
template <int NA, int D = 3>
struct StageBuf {
  float4 buf[kStages][NA][D * kChunk / 2];
};

// full[s]: the bulk copies of the chunk in stage s have landed (transaction
// count).  empty[s]: every warp has finished reading stage s (one arrival per
// warp).  abort: set by a thread whose wait expired.
struct Pipe {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  int abort;
};

__device__ __forceinline__ void pipe_init(Pipe& p, int warps) {
#pragma unroll
  for (int s = 0; s < kStages; ++s) {
    mbar_init(&p.full[s], 1);
    mbar_init(&p.empty[s], warps);
  }
  p.abort = 0;
  fence_mbar_init();
}

// Issue the bulk copies of chunk c (NA record arrays) into stage c % kStages.
// Source offsets and lengths are even, so records are copied whole.
template <int NA, int D>
__device__ __forceinline__ void issue_chunk(StageBuf<NA, D>& st, Pipe& pp, const float4* const* src, int j0, int j1,
                                            int c) {
  const int off = j0 + c * kChunk;
  const int len = min(kChunk, j1 - off);
  const unsigned bytes = static_cast<unsigned>(len) * (16 * D / 2);
  const int s = c % kStages;
  uint64_t* bar = &pp.full[s];
  mbar_arrive_expect_tx(bar, NA * bytes);
#pragma unroll
  for (int a = 0; a < NA; ++a) bulk_g2s(&st.buf[s][a][0], src[a] + (off / 2) * D, bytes, bar);
}

// Stream sources [j0, j1) through the stage ring.  Warp group `group` of
// `groups` consumes its share of each chunk: tile.consume(buffers, lo, hi)
// with [lo, hi) a contiguous piece, in multiples of 8 sources, of the chunk's
// sources.  The whole CTA calls this; thread 0 issues the copies.  Warps move on to the next chunk as soon as it has landed: a warp
// releases a stage through empty[s], and thread 0 refills a stage only after
// every warp has released it.  Returns false in every thread if a wait
// expired; the expiry is recorded in *status, and every copy still in flight
// has been waited for (bounded) before return.  Ends with a CTA barrier.
template <int NA, int Groups = 1, int D = 3, class Tile>
__device__ bool stream_sources(StageBuf<NA, D>& st, Pipe& pp, const float4* const* src, int j0, int j1, Tile& tile,
                               unsigned* status, int group = 0) {
  const int tid = threadIdx.x;
  const int nch = j1 > j0 ? (j1 - j0 + kChunk - 1) / kChunk : 0;
  int issued = 0;
  if (tid == 0) {
    for (; issued < nch && issued < kStages; ++issued) issue_chunk<NA, D>(st, pp, src, j0, j1, issued);
  }
  volatile int* abort = &pp.abort;
  for (int c = 0; c < nch; ++c) {
    const int s = c % kStages;
    if (*abort) break;
    if (!mbar_wait(&pp.full[s], (c / kStages) & 1)) {
      *abort = 1;
      break;
    }
    const float4* bufs[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) bufs[a] = st.buf[s][a];
    const int len = min(kChunk, j1 - (j0 + c * kChunk));
    if constexpr (Groups == 1) {
      tile.consume(bufs, 0, len);
    } else {
      const int piece = (len + kUnroll * Groups - 1) / (kUnroll * Groups) * kUnroll;
      const int lo = min(group * piece, len);
      tile.consume(bufs, lo, min(lo + piece, len));
    }
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(&pp.empty[s]);
    if (tid == 0 && c + kStages < nch) {
      // Refill stage s with chunk c + kStages once every warp has released it.
      if (mbar_wait(&pp.empty[s], (c / kStages) & 1)) {
        fence_proxy_async_smem();
        issue_chunk<NA, D>(st, pp, src, j0, j1, c + kStages);
        issued = c + kStages + 1;
      } else {
        *abort = 1;
      }
    }
  }
  __syncthreads();
  if (*abort) {
    if (tid == 0) {
      atomicOr(status, kErrTimeout);
      // Let every copy that was issued land before the CTA reuses or leaves
      // this memory: the last kStages chunks issued are the only ones that
      // can still be in flight.
      for (int d = max(0, issued - kStages); d < issued; ++d)
        (void)mbar_wait(&pp.full[d % kStages], (d / kStages) & 1);
    }
    __syncthreads();
    return false;
  }
  return true;
}

__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// Gaussian of two pairs at once from their squared prescaled distances.
__device__ __forceinline__ float2 gauss2(float2 r2) {
  return make_float2(ex2_approx(-r2.x), ex2_approx(-r2.y));
}

// Coordinate k (0..D-1) of landmark i from a pair-record array; field f
// selects the first (0) or second (1) quantity of the record.
template <int D = 3>
__device__ __forceinline__ float rec_get(const float4* rec, int i, int f, int k) {
  const float* r = reinterpret_cast<const float*>(rec + (i >> 1) * D);
  return __ldcg(r + 2 * D * f + 2 * k + (i & 1));
}

// The 2D float2 values of one pair record (D float4): value c < D is
// coordinate c of the first quantity, value D + c of the second, each for
// the record's two landmarks.
template <int D>
__device__ __forceinline__ void rec_split(const float4* rec, float2 (&v)[2 * D]) {
#pragma unroll
  for (int f = 0; f < D; ++f) {
    const float4 x = rec[f];
    v[2 * f] = lo2(x);
    v[2 * f + 1] = hi2(x);
  }
}

// ---------------------------------------------------------------- StepForward tile
// Per target i:  Hp_i = sum_j g_ij p_j  and  G~_i = sum_j c_ij g_ij (q~_i - q~_j),
// with Hq_i = -kappa G~_i.  D = 3 (or 2 for planar landmarks) coordinates.
template <int R, int D = 3>
struct FwdTile {
  float2 q[R][D], p[R][D];  // target, duplicated
  float sF[R][D], cF[R][D], sG[R][D], cG[R][D];

  __device__ __forceinline__ void load(const float4* qp, int base, int stride, int npad) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = base + r * stride;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float qk = i < npad ? -rec_get<D>(qp, i, 0, k) : 0.f;
        const float pk = i < npad ? rec_get<D>(qp, i, 1, k) : 0.f;
        q[r][k] = dup(qk);
        p[r][k] = dup(pk);
        sF[r][k] = cF[r][k] = sG[r][k] = cG[r][k] = 0.f;
      }
    }
  }

  // Sources [lo, hi) of the staged chunk; lo is a multiple of 8.
  __device__ __forceinline__ void consume(const float4* const* bufs, int lo, int hi) {
    const float4* Q = bufs[0];
    for (int sb = lo; sb < hi; sb += kSub) {
      const int sl = min(kSub, hi - sb);
      float2 aF[R][D], aG[R][D];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < D; ++k) aF[r][k] = aG[r][k] = make_float2(0.f, 0.f);
      for (int jj = 0; jj < sl; jj += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll / 2; ++u) {
          float2 v[2 * D];  // v[k] = -q~_j, v[D + k] = p_j
          rec_split<D>(Q + ((sb + jj) / 2 + u) * D, v);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            float2 d[D];
#pragma unroll
            for (int k = 0; k < D; ++k) d[k] = __fadd2_rn(q[r][k], v[k]);
            float2 r2 = __fmul2_rn(d[0], d[0]);
#pragma unroll
            for (int k = 1; k < D; ++k) r2 = __ffma2_rn(d[k], d[k], r2);
            const float2 g = gauss2(r2);
            float2 cc = __fmul2_rn(p[r][0], v[D]);
#pragma unroll
            for (int k = 1; k < D; ++k) cc = __ffma2_rn(p[r][k], v[D + k], cc);
            const float2 w = __fmul2_rn(g, cc);
#pragma unroll
            for (int k = 0; k < D; ++k) aF[r][k] = __ffma2_rn(g, v[D + k], aF[r][k]);
#pragma unroll
            for (int k = 0; k < D; ++k) aG[r][k] = __ffma2_rn(w, d[k], aG[r][k]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          kahan_add(sF[r][k], cF[r][k], __fadd_rn(aF[r][k].x, aF[r][k].y));
          kahan_add(sG[r][k], cG[r][k], __fadd_rn(aG[r][k].x, aG[r][k].y));
        }
    }
  }

  // out[0..D) = Hp, out[D..2D) = Hq of target r, as double-single values.
  __device__ __forceinline__ void result(int r, float kappa, ds out[2 * D]) const {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      out[k] = ds_from_kahan(sF[r][k], cF[r][k]);
      out[D + k] = ds_mul_f(ds_from_kahan(sG[r][k], cG[r][k]), -kappa);
    }
  }
};

// ---------------------------------------------------------------- StepBackward tile
// Sources carry q~ = kq q, p (QP records) and alpha, b~ = kappa beta (AB
// records).  Per pair:
//   d~ = q~_i - q~_j, g = 2^-|d~|^2, c = p_i.p_j, e~ = b~_i - b~_j,
//   t = e~.d~ (= s e.d), u = alpha_i.p_j + alpha_j.p_i, h = u + c t,
//   A1 += g c e~,  A2 += g h d~,  B += g (alpha_j + t p_j);
// dalpha = kq A1 - kappa A2 and dbeta = B.
template <int R, int D = 3>
struct BwdTile {
  float2 q[R][D], p[R][D], a[R][D], b[R][D];
  float s1[R][D], c1[R][D], s2[R][D], c2[R][D], sB[R][D], cB[R][D];

  __device__ __forceinline__ void load(const float4* qp, const float4* ab, int base, int stride, int npad) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = base + r * stride;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const bool in = i < npad;
        q[r][k] = dup(in ? -rec_get<D>(qp, i, 0, k) : 0.f);
        p[r][k] = dup(in ? rec_get<D>(qp, i, 1, k) : 0.f);
        a[r][k] = dup(in ? rec_get<D>(ab, i, 0, k) : 0.f);
        b[r][k] = dup(in ? -rec_get<D>(ab, i, 1, k) : 0.f);
        s1[r][k] = c1[r][k] = s2[r][k] = c2[r][k] = sB[r][k] = cB[r][k] = 0.f;
      }
    }
  }

  // Sources [lo, hi) of the staged chunk; lo is a multiple of 8.
  __device__ __forceinline__ void consume(const float4* const* bufs, int lo, int hi) {
    const float4* Q = bufs[0];
    const float4* Ab = bufs[1];
    for (int sb = lo; sb < hi; sb += kSub) {
      const int sl = min(kSub, hi - sb);
      float2 a1[R][D], a2[R][D], bb[R][D];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < D; ++k) a1[r][k] = a2[r][k] = bb[r][k] = make_float2(0.f, 0.f);
      for (int jj = 0; jj < sl; jj += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll / 2; ++u) {
          const int ri = ((sb + jj) / 2 + u) * D;
          float2 v[2 * D], w[2 * D];  // v: -q~_j, p_j;  w: alpha_j, -b~_j
          rec_split<D>(Q + ri, v);
          rec_split<D>(Ab + ri, w);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            float2 d[D], e[D];
#pragma unroll
            for (int k = 0; k < D; ++k) d[k] = __fadd2_rn(q[r][k], v[k]);
            float2 r2 = __fmul2_rn(d[0], d[0]);
#pragma unroll
            for (int k = 1; k < D; ++k) r2 = __ffma2_rn(d[k], d[k], r2);
            const float2 g = gauss2(r2);
            float2 cc = __fmul2_rn(p[r][0], v[D]);
#pragma unroll
            for (int k = 1; k < D; ++k) cc = __ffma2_rn(p[r][k], v[D + k], cc);
#pragma unroll
            for (int k = 0; k < D; ++k) e[k] = __fadd2_rn(b[r][k], w[D + k]);
            float2 t = __fmul2_rn(e[0], d[0]);
#pragma unroll
            for (int k = 1; k < D; ++k) t = __ffma2_rn(e[k], d[k], t);
            float2 uu = __fmul2_rn(a[r][0], v[D]);
#pragma unroll
            for (int k = 1; k < D; ++k) uu = __ffma2_rn(a[r][k], v[D + k], uu);
#pragma unroll
            for (int k = 0; k < D; ++k) uu = __ffma2_rn(w[k], p[r][k], uu);
            const float2 h = __ffma2_rn(cc, t, uu);
            const float2 gc = __fmul2_rn(g, cc);
            const float2 gh = __fmul2_rn(g, h);
#pragma unroll
            for (int k = 0; k < D; ++k) a1[r][k] = __ffma2_rn(gc, e[k], a1[r][k]);
#pragma unroll
            for (int k = 0; k < D; ++k) a2[r][k] = __ffma2_rn(gh, d[k], a2[r][k]);
#pragma unroll
            for (int k = 0; k < D; ++k) bb[r][k] = __ffma2_rn(g, __ffma2_rn(t, v[D + k], w[k]), bb[r][k]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          kahan_add(s1[r][k], c1[r][k], __fadd_rn(a1[r][k].x, a1[r][k].y));
          kahan_add(s2[r][k], c2[r][k], __fadd_rn(a2[r][k].x, a2[r][k].y));
          kahan_add(sB[r][k], cB[r][k], __fadd_rn(bb[r][k].x, bb[r][k].y));
        }
    }
  }

  // out[0..D) = dalpha, out[D..2D) = dbeta of target r.
  __device__ __forceinline__ void result(int r, float kq, float kappa, ds out[2 * D]) const {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      out[k] = ds_add(ds_mul_f(ds_from_kahan(s1[r][k], c1[r][k]), kq),
                      ds_mul_f(ds_from_kahan(s2[r][k], c2[r][k]), -kappa));
      out[D + k] = ds_from_kahan(sB[r][k], cB[r][k]);
    }
  }
};

}  // namespace gs
