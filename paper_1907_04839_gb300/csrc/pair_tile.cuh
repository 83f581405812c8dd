// Per-thread target tiles of the StepForward / StepBackward pair sums, and
// the TMA pipeline that streams a range of sources through shared memory.
// Both the split-partial kernels (pair_kernels.cu) and the fused step kernels
// (step_kernels.cu) are built from these pieces.
//
// A thread holds R targets in registers.  The targets of one CTA are
// tid + r*NT, r < R.  For each source staged in shared memory, every thread
// updates all of its R targets.  All threads of a warp read the same source
// at the same time, so the shared-memory load is a broadcast.  Sums are
// plain FP32 over a sub-block of at most kSub sources, then folded into a
// Kahan (sum, compensation) pair.
#pragma once

#include "gs_device.cuh"
#include "gs_internal.h"

namespace gs {

constexpr int kSub = 64;    // sources per plain-FP32 sub-block before a Kahan fold
constexpr int kUnroll = 8;  // split lengths are multiples of this

// Two chunk buffers for NA source arrays.  The mbarriers live outside, so
// this memory can be reused once the last chunk has been consumed.
template <int NA>
struct StageBuf {
  float4 buf[2][NA][kChunk];
};

__device__ __forceinline__ void stage_init(uint64_t* full) {
  mbar_init(&full[0], 1);
  mbar_init(&full[1], 1);
  fence_mbar_init();
}

// Issue the bulk copies of chunk c (NA arrays) into buffer c & 1.
template <int NA>
__device__ __forceinline__ void issue_chunk(StageBuf<NA>& st, uint64_t* full, const float4* const* src, int j0,
                                            int j1, int c) {
  const int off = j0 + c * kChunk;
  const int len = min(kChunk, j1 - off);
  const unsigned bytes = static_cast<unsigned>(len) * sizeof(float4);
  uint64_t* bar = &full[c & 1];
  mbar_arrive_expect_tx(bar, NA * bytes);
#pragma unroll
  for (int a = 0; a < NA; ++a) bulk_g2s(&st.buf[c & 1][a][0], src[a] + off, bytes, bar);
}

// Stream sources [j0, j1) through the double buffer and feed each chunk to
// tile.consume(buffers, len).  The whole CTA calls this.  Returns false in
// every thread if a wait expired; the expiry is recorded in *status, and
// every copy still in flight has been waited for (bounded) before return.
template <int NA, class Tile>
__device__ bool stream_sources(StageBuf<NA>& st, uint64_t* full, const float4* const* src, int j0, int j1,
                               Tile& tile, unsigned* status) {
  const int tid = threadIdx.x;
  const int nch = (j1 - j0 + kChunk - 1) / kChunk;
  int issued = 0;
  if (tid == 0 && nch > 0) {
    issue_chunk<NA>(st, full, src, j0, j1, 0);
    issued = 1;
    if (nch > 1) {
      issue_chunk<NA>(st, full, src, j0, j1, 1);
      issued = 2;
    }
  }
  int c = 0;
  for (; c < nch; ++c) {
    const int b = c & 1;
    const bool ok = mbar_wait(&full[b], (c >> 1) & 1);
    const int len = min(kChunk, j1 - (j0 + c * kChunk));
    const float4* bufs[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) bufs[a] = st.buf[b][a];
    tile.consume(bufs, len);
    // Every thread is done with buffer b; a uniform vote on the wait result.
    if (__syncthreads_or(!ok)) break;
    if (tid == 0 && c + 2 < nch) {
      fence_proxy_async_smem();
      issue_chunk<NA>(st, full, src, j0, j1, c + 2);
      issued = c + 3;
    }
  }
  if (c < nch) {
    if (tid == 0) {
      atomicOr(status, kErrTimeout);
      for (int d = c; d < issued; ++d) (void)mbar_wait(&full[d & 1], (d >> 1) & 1);
    }
    __syncthreads();
    return false;
  }
  return true;
}

// ---------------------------------------------------------------- StepForward tile
// Per target i:  Hp_i = sum_j g_ij p_j  and  G~_i = sum_j c_ij g_ij (q~_i - q~_j),
// with Hq_i = -kappa G~_i.
template <int R>
struct FwdTile {
  float qx[R], qy[R], qz[R], px[R], py[R], pz[R];
  float sF[R][3], cF[R][3], sG[R][3], cG[R][3];

  __device__ __forceinline__ void load(const float4* q4, const float4* p4, int base, int stride, int npad) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = base + r * stride;
      float4 qi = make_float4(0.f, 0.f, 0.f, 0.f), pi = qi;
      if (i < npad) {
        qi = q4[i];
        pi = p4[i];
      }
      qx[r] = qi.x; qy[r] = qi.y; qz[r] = qi.z;
      px[r] = pi.x; py[r] = pi.y; pz[r] = pi.z;
#pragma unroll
      for (int k = 0; k < 3; ++k) sF[r][k] = cF[r][k] = sG[r][k] = cG[r][k] = 0.f;
    }
  }

  __device__ __forceinline__ void consume(const float4* const* bufs, int len) {
    const float4* Q = bufs[0];
    const float4* P = bufs[1];
    for (int sb = 0; sb < len; sb += kSub) {
      const int sl = min(kSub, len - sb);
      float aF[R][3], aG[R][3];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) aF[r][k] = aG[r][k] = 0.f;
      for (int jj = 0; jj < sl; jj += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const float4 qj = Q[sb + jj + u];
          const float4 pj = P[sb + jj + u];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float dx = qx[r] - qj.x, dy = qy[r] - qj.y, dz = qz[r] - qj.z;
            const float nr = fmaf(-dz, dz, fmaf(-dy, dy, -dx * dx));
            const float g = ex2_approx(nr);
            const float cc = fmaf(pz[r], pj.z, fmaf(py[r], pj.y, px[r] * pj.x));
            const float w = g * cc;
            aF[r][0] = fmaf(g, pj.x, aF[r][0]);
            aF[r][1] = fmaf(g, pj.y, aF[r][1]);
            aF[r][2] = fmaf(g, pj.z, aF[r][2]);
            aG[r][0] = fmaf(w, dx, aG[r][0]);
            aG[r][1] = fmaf(w, dy, aG[r][1]);
            aG[r][2] = fmaf(w, dz, aG[r][2]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          kahan_add(sF[r][k], cF[r][k], aF[r][k]);
          kahan_add(sG[r][k], cG[r][k], aG[r][k]);
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
// Sources carry q~ = kq q, p, alpha and b~ = kappa beta.  Per pair:
//   d~ = q~_i - q~_j, g = 2^-|d~|^2, c = p_i.p_j, e~ = b~_i - b~_j,
//   t = e~.d~ (= s e.d), u = alpha_i.p_j + alpha_j.p_i, h = u + c t,
//   A1 += g c e~,  A2 += g h d~,  B += g (alpha_j + t p_j);
// dalpha = kq A1 - kappa A2 and dbeta = B.
template <int R>
struct BwdTile {
  float qx[R], qy[R], qz[R], px[R], py[R], pz[R], ax[R], ay[R], az[R], bx[R], by[R], bz[R];
  float s1[R][3], c1[R][3], s2[R][3], c2[R][3], sB[R][3], cB[R][3];

  __device__ __forceinline__ void load(const float4* q4, const float4* p4, const float4* a4, const float4* b4,
                                       int base, int stride, int npad) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = base + r * stride;
      float4 qi = make_float4(0.f, 0.f, 0.f, 0.f), pi = qi, ai = qi, bi = qi;
      if (i < npad) {
        qi = q4[i];
        pi = p4[i];
        ai = a4[i];
        bi = b4[i];
      }
      qx[r] = qi.x; qy[r] = qi.y; qz[r] = qi.z;
      px[r] = pi.x; py[r] = pi.y; pz[r] = pi.z;
      ax[r] = ai.x; ay[r] = ai.y; az[r] = ai.z;
      bx[r] = bi.x; by[r] = bi.y; bz[r] = bi.z;
#pragma unroll
      for (int k = 0; k < 3; ++k) s1[r][k] = c1[r][k] = s2[r][k] = c2[r][k] = sB[r][k] = cB[r][k] = 0.f;
    }
  }

  __device__ __forceinline__ void consume(const float4* const* bufs, int len) {
    const float4* Q = bufs[0];
    const float4* P = bufs[1];
    const float4* A = bufs[2];
    const float4* B = bufs[3];
    for (int sb = 0; sb < len; sb += kSub) {
      const int sl = min(kSub, len - sb);
      float a1[R][3], a2[R][3], bb[R][3];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) a1[r][k] = a2[r][k] = bb[r][k] = 0.f;
      for (int jj = 0; jj < sl; jj += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const float4 qj = Q[sb + jj + u];
          const float4 pj = P[sb + jj + u];
          const float4 aj = A[sb + jj + u];
          const float4 bj = B[sb + jj + u];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float dx = qx[r] - qj.x, dy = qy[r] - qj.y, dz = qz[r] - qj.z;
            const float nr = fmaf(-dz, dz, fmaf(-dy, dy, -dx * dx));
            const float g = ex2_approx(nr);
            const float cc = fmaf(pz[r], pj.z, fmaf(py[r], pj.y, px[r] * pj.x));
            const float ex = bx[r] - bj.x, ey = by[r] - bj.y, ez = bz[r] - bj.z;
            const float t = fmaf(ez, dz, fmaf(ey, dy, ex * dx));
            float uu = ax[r] * pj.x;
            uu = fmaf(ay[r], pj.y, uu);
            uu = fmaf(az[r], pj.z, uu);
            uu = fmaf(aj.x, px[r], uu);
            uu = fmaf(aj.y, py[r], uu);
            uu = fmaf(aj.z, pz[r], uu);
            const float h = fmaf(cc, t, uu);
            const float gc = g * cc;
            const float gh = g * h;
            a1[r][0] = fmaf(gc, ex, a1[r][0]);
            a1[r][1] = fmaf(gc, ey, a1[r][1]);
            a1[r][2] = fmaf(gc, ez, a1[r][2]);
            a2[r][0] = fmaf(gh, dx, a2[r][0]);
            a2[r][1] = fmaf(gh, dy, a2[r][1]);
            a2[r][2] = fmaf(gh, dz, a2[r][2]);
            bb[r][0] = fmaf(g, fmaf(t, pj.x, aj.x), bb[r][0]);
            bb[r][1] = fmaf(g, fmaf(t, pj.y, aj.y), bb[r][1]);
            bb[r][2] = fmaf(g, fmaf(t, pj.z, aj.z), bb[r][2]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          kahan_add(s1[r][k], c1[r][k], a1[r][k]);
          kahan_add(s2[r][k], c2[r][k], a2[r][k]);
          kahan_add(sB[r][k], cB[r][k], bb[r][k]);
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
