// Pair-sum kernels: StepForward and StepBackward (Section 2.2, 2.5).
//
// These sums are the O(N^2) hot path of the method.  The paper's Algorithm 4
// has one block per target, a shared-memory tree reduction over 256 sources
// and atomicAdd into global memory.  This design differs:
//  * A CTA owns a tile of NT*R targets, held in registers (R per thread).
//  * A CTA streams one contiguous range of sources (a "split") through shared
//    memory.  The staging uses bulk TMA copies (cp.async.bulk) into a double
//    buffer, and each buffer is guarded by an mbarrier.
//  * Every warp reads the same source at the same time, so the shared-memory
//    read is a broadcast.
//  * Each thread accumulates plain FP32 over a sub-block of at most 64
//    sources, then folds the sub-block sum into a Kahan (sum, compensation)
//    pair.  This is the compensated accumulation that the paper's accuracy
//    argument (Section 2.2) asks for.
//  * The split's result goes out as a double-single partial per target.  No
//    atomics are used, so the result is deterministic.  A separate kernel
//    combines the splits in a fixed order (combine.cu).
//  * The Gaussian is a single MUFU ex2 on prescaled coordinates.  With
//    q~ = kq q and kq^2 = log2(e) / (2 sigma^2),
//    g = exp(-|d|^2 / (2 sigma^2)) = 2^(-|q~_i - q~_j|^2).
//  * The kernels use no tensor cores.  The pair work is not a dense
//    contraction (d = 3), and it is bound by the FP32 pipe.
#include <cstdio>

#include "gs_device.cuh"
#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kSub = 64;    // sources per plain-FP32 sub-block before a Kahan fold
constexpr int kUnroll = 8;  // split lengths are multiples of this

// Shared staging for NA source arrays, two chunks deep.
template <int NA>
struct Stage {
  float4 buf[2][NA][kChunk];
  uint64_t full[2];
  int abort;
};

// Issue the bulk copies of chunk c (NA arrays) into buffer c & 1.
template <int NA>
__device__ __forceinline__ void issue_chunk(Stage<NA>& st, const float4* const* src, int j0, int j1, int c) {
  const int off = j0 + c * kChunk;
  const int len = min(kChunk, j1 - off);
  const unsigned bytes = static_cast<unsigned>(len) * sizeof(float4);
  uint64_t* bar = &st.full[c & 1];
  mbar_arrive_expect_tx(bar, NA * bytes);
#pragma unroll
  for (int a = 0; a < NA; ++a) bulk_g2s(&st.buf[c & 1][a][0], src[a] + off, bytes, bar);
}

// After an expired wait: wait (bounded) for every copy still in flight so the
// CTA never exits with a bulk copy writing into its shared memory.
template <int NA>
__device__ __forceinline__ void drain(Stage<NA>& st, int consumed, int issued) {
  for (int c = consumed; c < issued; ++c) (void)mbar_wait(&st.full[c & 1], (c >> 1) & 1);
}

}  // namespace

// ---------------------------------------------------------------- StepForward
// Per target i and split [j0, j1):
//   Hp_i  = sum_j g_ij p_j
//   G~_i  = sum_j c_ij g_ij (q~_i - q~_j),   Hq_i = -kappa G~_i
template <int NT, int R>
__global__ void __launch_bounds__(NT) k_pair_forward(PairFwdArgs a) {
  __shared__ __align__(128) Stage<2> st;
  const int tid = threadIdx.x;
  const int j0 = blockIdx.y * a.split_len;
  const int j1 = min(j0 + a.split_len, a.npad);
  const int nch = (j1 - j0 + kChunk - 1) / kChunk;

  if (tid == 0) {
    mbar_init(&st.full[0], 1);
    mbar_init(&st.full[1], 1);
    fence_mbar_init();
    st.abort = 0;
  }
  __syncthreads();
  pdl_wait();  // the previous step's state must be complete
  pdl_launch_dependents();

  const float4* src[2] = {a.q4, a.p4};
  int issued = 0;
  if (tid == 0 && nch > 0) {
    issue_chunk<2>(st, src, j0, j1, 0);
    issued = 1;
    if (nch > 1) { issue_chunk<2>(st, src, j0, j1, 1); issued = 2; }
  }

  float qx[R], qy[R], qz[R], px[R], py[R], pz[R];
  const int base = blockIdx.x * (NT * R) + tid;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = base + r * NT;
    float4 qi = make_float4(0.f, 0.f, 0.f, 0.f), pi = qi;
    if (i < a.npad) { qi = a.q4[i]; pi = a.p4[i]; }
    qx[r] = qi.x; qy[r] = qi.y; qz[r] = qi.z;
    px[r] = pi.x; py[r] = pi.y; pz[r] = pi.z;
  }
  float sF[R][3], cF[R][3], sG[R][3], cG[R][3];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) sF[r][k] = cF[r][k] = sG[r][k] = cG[r][k] = 0.f;

  int c = 0;
  for (; c < nch; ++c) {
    const int b = c & 1;
    const bool ok = mbar_wait(&st.full[b], (c >> 1) & 1);
    const int len = min(kChunk, j1 - (j0 + c * kChunk));
    const float4* Q = st.buf[b][0];
    const float4* P = st.buf[b][1];
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
    // Every thread is done with buffer b; a uniform vote on the wait result.
    if (__syncthreads_or(!ok)) break;
    if (tid == 0 && c + 2 < nch) {
      fence_proxy_async_smem();
      issue_chunk<2>(st, src, j0, j1, c + 2);
      issued = c + 3;
    }
  }
  if (c < nch) {  // a wait expired: record it, let copies land, write nothing
    if (tid == 0) {
      atomicOr(a.status, kErrTimeout);
      drain<2>(st, c, issued);
    }
    return;
  }

  const float kap = a.kappa;
  Partial* out = a.part + static_cast<size_t>(blockIdx.y) * a.npad;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = base + r * NT;
    if (i >= a.npad) continue;
    Partial pt;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const ds hp = ds_from_kahan(sF[r][k], cF[r][k]);
      const ds hq = ds_mul_f(ds_from_kahan(sG[r][k], cG[r][k]), -kap);
      pt.c[k] = make_float2(hp.hi, hp.lo);
      pt.c[3 + k] = make_float2(hq.hi, hq.lo);
    }
    out[i] = pt;
  }
}

// ---------------------------------------------------------------- StepBackward
// Sources carry q~ = kq q, p, alpha and b~ = kappa beta.  Per pair:
//   d~ = q~_i - q~_j, g = 2^-|d~|^2, c = p_i.p_j, e~ = b~_i - b~_j,
//   t = e~.d~ (= s e.d), u = alpha_i.p_j + alpha_j.p_i, h = u + c t,
//   A1 += g c e~,  A2 += g h d~,  B += g (alpha_j + t p_j);
// dalpha = kq A1 - kappa A2 and dbeta = B.
template <int NT, int R>
__global__ void __launch_bounds__(NT) k_pair_backward(PairBwdArgs a) {
  __shared__ __align__(128) Stage<4> st;
  const int tid = threadIdx.x;
  const int j0 = blockIdx.y * a.split_len;
  const int j1 = min(j0 + a.split_len, a.npad);
  const int nch = (j1 - j0 + kChunk - 1) / kChunk;

  if (tid == 0) {
    mbar_init(&st.full[0], 1);
    mbar_init(&st.full[1], 1);
    fence_mbar_init();
    st.abort = 0;
  }
  __syncthreads();
  pdl_wait();
  pdl_launch_dependents();

  const float4* src[4] = {a.q4, a.p4, a.a4, a.b4};
  int issued = 0;
  if (tid == 0 && nch > 0) {
    issue_chunk<4>(st, src, j0, j1, 0);
    issued = 1;
    if (nch > 1) { issue_chunk<4>(st, src, j0, j1, 1); issued = 2; }
  }

  float qx[R], qy[R], qz[R], px[R], py[R], pz[R], ax[R], ay[R], az[R], bx[R], by[R], bz[R];
  const int base = blockIdx.x * (NT * R) + tid;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = base + r * NT;
    float4 qi = make_float4(0.f, 0.f, 0.f, 0.f), pi = qi, ai = qi, bi = qi;
    if (i < a.npad) { qi = a.q4[i]; pi = a.p4[i]; ai = a.a4[i]; bi = a.b4[i]; }
    qx[r] = qi.x; qy[r] = qi.y; qz[r] = qi.z;
    px[r] = pi.x; py[r] = pi.y; pz[r] = pi.z;
    ax[r] = ai.x; ay[r] = ai.y; az[r] = ai.z;
    bx[r] = bi.x; by[r] = bi.y; bz[r] = bi.z;
  }
  // Kahan state for A1, A2, B per target.
  float s1[R][3], c1[R][3], s2[R][3], c2[R][3], sB[R][3], cB[R][3];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) s1[r][k] = c1[r][k] = s2[r][k] = c2[r][k] = sB[r][k] = cB[r][k] = 0.f;

  int c = 0;
  for (; c < nch; ++c) {
    const int b = c & 1;
    const bool ok = mbar_wait(&st.full[b], (c >> 1) & 1);
    const int len = min(kChunk, j1 - (j0 + c * kChunk));
    const float4* Q = st.buf[b][0];
    const float4* P = st.buf[b][1];
    const float4* A = st.buf[b][2];
    const float4* B = st.buf[b][3];
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
    if (__syncthreads_or(!ok)) break;
    if (tid == 0 && c + 2 < nch) {
      fence_proxy_async_smem();
      issue_chunk<4>(st, src, j0, j1, c + 2);
      issued = c + 3;
    }
  }
  if (c < nch) {
    if (tid == 0) {
      atomicOr(a.status, kErrTimeout);
      drain<4>(st, c, issued);
    }
    return;
  }

  Partial* out = a.part + static_cast<size_t>(blockIdx.y) * a.npad;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = base + r * NT;
    if (i >= a.npad) continue;
    Partial pt;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const ds da = ds_add(ds_mul_f(ds_from_kahan(s1[r][k], c1[r][k]), a.kq),
                           ds_mul_f(ds_from_kahan(s2[r][k], c2[r][k]), -a.kappa));
      const ds db = ds_from_kahan(sB[r][k], cB[r][k]);
      pt.c[k] = make_float2(da.hi, da.lo);
      pt.c[3 + k] = make_float2(db.hi, db.lo);
    }
    out[i] = pt;
  }
}

// ---------------------------------------------------------------- host side

namespace {

constexpr int kFwdNT = 64, kFwdR = 4;
constexpr int kBwdNT = 64, kBwdR = 2;

// Pick the number of source splits so that tiles * splits fills every SM
// with `per_sm` resident CTAs, with split lengths a multiple of kUnroll.
PairConfig make_config(int npad, int num_sms, int threads, int R, int per_sm) {
  PairConfig c;
  c.threads = threads;
  c.R = R;
  const int tile = threads * R;
  c.tiles = (npad + tile - 1) / tile;
  const int want = num_sms * per_sm;
  int splits = (want + c.tiles - 1) / c.tiles;
  splits = max(1, min(splits, npad / kUnroll));
  int len = (npad + splits - 1) / splits;
  len = (len + kUnroll - 1) / kUnroll * kUnroll;
  c.split_len = len;
  c.splits = (npad + len - 1) / len;
  return c;
}

template <typename K, typename A>
cudaError_t launch(K kern, dim3 grid, dim3 block, const A& args, cudaStream_t st, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args);
}

}  // namespace

PairConfig choose_forward_config(int npad, int num_sms) {
  return make_config(npad, num_sms, kFwdNT, kFwdR, 8);
}

PairConfig choose_forward_config_capped(int npad, int num_sms, int max_splits) {
  PairConfig c = make_config(npad, num_sms, kFwdNT, kFwdR, 8);
  if (c.splits > max_splits) {
    int len = (npad + max_splits - 1) / max_splits;
    len = (len + kUnroll - 1) / kUnroll * kUnroll;
    c.split_len = len;
    c.splits = (npad + len - 1) / len;
  }
  return c;
}

PairConfig choose_backward_config(int npad, int num_sms) {
  return make_config(npad, num_sms, kBwdNT, kBwdR, 8);
}

cudaError_t launch_pair_forward(const PairConfig& cfg, const PairFwdArgs& a, cudaStream_t st, bool pdl) {
  if (cfg.threads != kFwdNT || cfg.R != kFwdR) return cudaErrorInvalidValue;
  return launch(k_pair_forward<kFwdNT, kFwdR>, dim3(cfg.tiles, cfg.splits), dim3(kFwdNT), a, st, pdl);
}

cudaError_t launch_pair_backward(const PairConfig& cfg, const PairBwdArgs& a, cudaStream_t st, bool pdl) {
  if (cfg.threads != kBwdNT || cfg.R != kBwdR) return cudaErrorInvalidValue;
  return launch(k_pair_backward<kBwdNT, kBwdR>, dim3(cfg.tiles, cfg.splits), dim3(kBwdNT), a, st, pdl);
}

}  // namespace gs
