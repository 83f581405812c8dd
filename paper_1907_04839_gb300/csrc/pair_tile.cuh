// Per-thread target tiles of the StepForward / StepBackward pair sums, and
// the TMA pipeline that streams a range of sources through shared memory.
// Both the split-partial kernels (pair_kernels.cu) and the fused step kernels
// (step_kernels.cu) are built from these pieces.
//
// Packed arithmetic.  Sources sit in memory as pair records: two landmarks
// interleaved per coordinate (layout in gs_internal.h).  The inner loop uses
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

constexpr int kSub = 64;    // sources per plain-FP32 sub-block before a Kahan fold
constexpr int kUnroll = 8;  // split lengths are multiples of this

// kStages chunk buffers for NA record arrays (kChunk sources = kChunk/2
// records of 3 float4 each).  The mbarriers live outside (struct Pipe), so
// this memory can be reused once the last chunk has been consumed.
template <int NA>
struct StageBuf {
  float4 buf[kStages][NA][kRecF4 * kChunk / 2];
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
template <int NA>
__device__ __forceinline__ void issue_chunk(StageBuf<NA>& st, Pipe& pp, const float4* const* src, int j0, int j1,
                                            int c) {
  const int off = j0 + c * kChunk;
  const int len = min(kChunk, j1 - off);
  const unsigned bytes = static_cast<unsigned>(len) * (kRecBytes / 2);
  const int s = c % kStages;
  uint64_t* bar = &pp.full[s];
  mbar_arrive_expect_tx(bar, NA * bytes);
#pragma unroll
  for (int a = 0; a < NA; ++a) bulk_g2s(&st.buf[s][a][0], src[a] + (off / 2) * kRecF4, bytes, bar);
}

// Stream sources [j0, j1) through the stage ring.  Warp group `group` of
// `groups` consumes its share of each chunk: tile.consume(buffers, lo, hi)
// with [lo, hi) a contiguous piece, in multiples of 8 sources, of the chunk's
// sources.  The whole CTA calls this; thread 0 issues the copies.  Warps move on to the next chunk as soon as it has landed: a warp
// releases a stage through empty[s], and thread 0 refills a stage only after
// every warp has released it.  Returns false in every thread if a wait
// expired; the expiry is recorded in *status, and every copy still in flight
// has been waited for (bounded) before return.  Ends with a CTA barrier.
template <int NA, int Groups = 1, class Tile>
__device__ bool stream_sources(StageBuf<NA>& st, Pipe& pp, const float4* const* src, int j0, int j1, Tile& tile,
                               unsigned* status, int group = 0) {
  const int tid = threadIdx.x;
  const int nch = j1 > j0 ? (j1 - j0 + kChunk - 1) / kChunk : 0;
  int issued = 0;
  if (tid == 0) {
    for (; issued < nch && issued < kStages; ++issued) issue_chunk<NA>(st, pp, src, j0, j1, issued);
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
        issue_chunk<NA>(st, pp, src, j0, j1, c + kStages);
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

// Coordinate k (0..2) of landmark i from a pair-record array; field f selects
// the first (0) or second (1) quantity of the record.
__device__ __forceinline__ float rec_get(const float4* rec, int i, int f, int k) {
  const float* r = reinterpret_cast<const float*>(rec + (i >> 1) * kRecF4);
  return __ldcg(r + 6 * f + 2 * k + (i & 1));
}

// ---------------------------------------------------------------- StepForward tile
// Per target i:  Hp_i = sum_j g_ij p_j  and  G~_i = sum_j c_ij g_ij (q~_i - q~_j),
// with Hq_i = -kappa G~_i.
template <int R>
struct FwdTile {
  float2 qx[R], qy[R], qz[R], px[R], py[R], pz[R];  // target, duplicated
  float sF[R][3], cF[R][3], sG[R][3], cG[R][3];

  __device__ __forceinline__ void load(const float4* qp, int base, int stride, int npad) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = base + r * stride;
      float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (i < npad) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          v[k] = -rec_get(qp, i, 0, k);
          v[3 + k] = rec_get(qp, i, 1, k);
        }
      }
      qx[r] = dup(v[0]); qy[r] = dup(v[1]); qz[r] = dup(v[2]);
      px[r] = dup(v[3]); py[r] = dup(v[4]); pz[r] = dup(v[5]);
#pragma unroll
      for (int k = 0; k < 3; ++k) sF[r][k] = cF[r][k] = sG[r][k] = cG[r][k] = 0.f;
    }
  }

  // Sources [lo, hi) of the staged chunk; lo is a multiple of 8.
  __device__ __forceinline__ void consume(const float4* const* bufs, int lo, int hi) {
    const float4* Q = bufs[0];
    for (int sb = lo; sb < hi; sb += kSub) {
      const int sl = min(kSub, hi - sb);
      float2 aF[R][3], aG[R][3];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) aF[r][k] = aG[r][k] = make_float2(0.f, 0.f);
      for (int jj = 0; jj < sl; jj += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll / 2; ++u) {
          const float4* rec = Q + ((sb + jj) / 2 + u) * kRecF4;
          const float4 A = rec[0], B = rec[1], C = rec[2];
          const float2 nqx = lo2(A), nqy = hi2(A), nqz = lo2(B);
          const float2 pjx = hi2(B), pjy = lo2(C), pjz = hi2(C);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float2 dx = __fadd2_rn(qx[r], nqx);
            const float2 dy = __fadd2_rn(qy[r], nqy);
            const float2 dz = __fadd2_rn(qz[r], nqz);
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            const float2 g = gauss2(r2);
            float2 cc = __fmul2_rn(px[r], pjx);
            cc = __ffma2_rn(py[r], pjy, cc);
            cc = __ffma2_rn(pz[r], pjz, cc);
            const float2 w = __fmul2_rn(g, cc);
            aF[r][0] = __ffma2_rn(g, pjx, aF[r][0]);
            aF[r][1] = __ffma2_rn(g, pjy, aF[r][1]);
            aF[r][2] = __ffma2_rn(g, pjz, aF[r][2]);
            aG[r][0] = __ffma2_rn(w, dx, aG[r][0]);
            aG[r][1] = __ffma2_rn(w, dy, aG[r][1]);
            aG[r][2] = __ffma2_rn(w, dz, aG[r][2]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          kahan_add(sF[r][k], cF[r][k], __fadd_rn(aF[r][k].x, aF[r][k].y));
          kahan_add(sG[r][k], cG[r][k], __fadd_rn(aG[r][k].x, aG[r][k].y));
        }
    }
  }

  // out[0..2] = Hp, out[3..5] = Hq of target r, as double-single values.
  __device__ __forceinline__ void result(int r, float kappa, ds out[6]) const {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      out[k] = ds_from_kahan(sF[r][k], cF[r][k]);
      out[3 + k] = ds_mul_f(ds_from_kahan(sG[r][k], cG[r][k]), -kappa);
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
template <int R>
struct BwdTile {
  float2 qx[R], qy[R], qz[R], px[R], py[R], pz[R], ax[R], ay[R], az[R], bx[R], by[R], bz[R];
  float s1[R][3], c1[R][3], s2[R][3], c2[R][3], sB[R][3], cB[R][3];

  __device__ __forceinline__ void load(const float4* qp, const float4* ab, int base, int stride, int npad) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = base + r * stride;
      float v[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = 0.f;
      if (i < npad) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          v[k] = -rec_get(qp, i, 0, k);
          v[3 + k] = rec_get(qp, i, 1, k);
          v[6 + k] = rec_get(ab, i, 0, k);
          v[9 + k] = -rec_get(ab, i, 1, k);
        }
      }
      qx[r] = dup(v[0]); qy[r] = dup(v[1]); qz[r] = dup(v[2]);
      px[r] = dup(v[3]); py[r] = dup(v[4]); pz[r] = dup(v[5]);
      ax[r] = dup(v[6]); ay[r] = dup(v[7]); az[r] = dup(v[8]);
      bx[r] = dup(v[9]); by[r] = dup(v[10]); bz[r] = dup(v[11]);
#pragma unroll
      for (int k = 0; k < 3; ++k) s1[r][k] = c1[r][k] = s2[r][k] = c2[r][k] = sB[r][k] = cB[r][k] = 0.f;
    }
  }

  // Sources [lo, hi) of the staged chunk; lo is a multiple of 8.
  __device__ __forceinline__ void consume(const float4* const* bufs, int lo, int hi) {
    const float4* Q = bufs[0];
    const float4* Ab = bufs[1];
    for (int sb = lo; sb < hi; sb += kSub) {
      const int sl = min(kSub, hi - sb);
      float2 a1[R][3], a2[R][3], bb[R][3];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) a1[r][k] = a2[r][k] = bb[r][k] = make_float2(0.f, 0.f);
      for (int jj = 0; jj < sl; jj += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll / 2; ++u) {
          const int ri = ((sb + jj) / 2 + u) * kRecF4;
          const float4 A = Q[ri], B = Q[ri + 1], C = Q[ri + 2];
          const float4 D = Ab[ri], E = Ab[ri + 1], F = Ab[ri + 2];
          const float2 nqx = lo2(A), nqy = hi2(A), nqz = lo2(B);
          const float2 pjx = hi2(B), pjy = lo2(C), pjz = hi2(C);
          const float2 ajx = lo2(D), ajy = hi2(D), ajz = lo2(E);
          const float2 nbx = hi2(E), nby = lo2(F), nbz = hi2(F);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float2 dx = __fadd2_rn(qx[r], nqx);
            const float2 dy = __fadd2_rn(qy[r], nqy);
            const float2 dz = __fadd2_rn(qz[r], nqz);
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            const float2 g = gauss2(r2);
            float2 cc = __fmul2_rn(px[r], pjx);
            cc = __ffma2_rn(py[r], pjy, cc);
            cc = __ffma2_rn(pz[r], pjz, cc);
            const float2 ex = __fadd2_rn(bx[r], nbx);
            const float2 ey = __fadd2_rn(by[r], nby);
            const float2 ez = __fadd2_rn(bz[r], nbz);
            float2 t = __fmul2_rn(ex, dx);
            t = __ffma2_rn(ey, dy, t);
            t = __ffma2_rn(ez, dz, t);
            float2 uu = __fmul2_rn(ax[r], pjx);
            uu = __ffma2_rn(ay[r], pjy, uu);
            uu = __ffma2_rn(az[r], pjz, uu);
            uu = __ffma2_rn(ajx, px[r], uu);
            uu = __ffma2_rn(ajy, py[r], uu);
            uu = __ffma2_rn(ajz, pz[r], uu);
            const float2 h = __ffma2_rn(cc, t, uu);
            const float2 gc = __fmul2_rn(g, cc);
            const float2 gh = __fmul2_rn(g, h);
            a1[r][0] = __ffma2_rn(gc, ex, a1[r][0]);
            a1[r][1] = __ffma2_rn(gc, ey, a1[r][1]);
            a1[r][2] = __ffma2_rn(gc, ez, a1[r][2]);
            a2[r][0] = __ffma2_rn(gh, dx, a2[r][0]);
            a2[r][1] = __ffma2_rn(gh, dy, a2[r][1]);
            a2[r][2] = __ffma2_rn(gh, dz, a2[r][2]);
            bb[r][0] = __ffma2_rn(g, __ffma2_rn(t, pjx, ajx), bb[r][0]);
            bb[r][1] = __ffma2_rn(g, __ffma2_rn(t, pjy, ajy), bb[r][1]);
            bb[r][2] = __ffma2_rn(g, __ffma2_rn(t, pjz, ajz), bb[r][2]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          kahan_add(s1[r][k], c1[r][k], __fadd_rn(a1[r][k].x, a1[r][k].y));
          kahan_add(s2[r][k], c2[r][k], __fadd_rn(a2[r][k].x, a2[r][k].y));
          kahan_add(sB[r][k], cB[r][k], __fadd_rn(bb[r][k].x, bb[r][k].y));
        }
    }
  }

  // out[0..2] = dalpha, out[3..5] = dbeta of target r.
  __device__ __forceinline__ void result(int r, float kq, float kappa, ds out[6]) const {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      out[k] = ds_add(ds_mul_f(ds_from_kahan(s1[r][k], c1[r][k]), kq),
                      ds_mul_f(ds_from_kahan(s2[r][k], c2[r][k]), -kappa));
      out[3 + k] = ds_from_kahan(sB[r][k], cB[r][k]);
    }
  }
};

}  // namespace gs
