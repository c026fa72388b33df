// Slice-tiled Jacobi COCG/CG iteration: three launches and ten vector passes
// per Krylov iteration, every inner product computed directly from the
// vectors it is defined by (the textbook recurrences).
//
// Notation: L = the step operator of Appendix B (lab frame) or Appendix A
// (transformed frame), D = diag(L) (complex per system; real for CG), and
// (a, b) the unconjugated bilinear form (COCG, lab frame) or a^H b (CG,
// transformed frame).  Iteration k:
//   spmm:   q = L p,  alpha = rho / (p, q)                 p gathered, q written
//   update: r -= alpha q,  z = D^-1 r,  rho' = (r, z),  |r|^2,  beta = rho'/rho
//                                                          r, q read, r written
//   xp:     x += alpha p,  p = D^-1 r + beta p             x, p, r read, x, p written
// The x update rides on the p update (both read p), which is where the ten
// passes come from (the row variant's eleven read p twice).  One-reduction
// rearrangements (the rho' expansion, Chronopoulos-Gear) were tried and lose
// too much accuracy for the complex symmetric COCG of the lab frame, whose
// bilinear forms cancel strongly.
//
// SpMM layout.  Rows are grouped into Morton tiles (HaloTiles, owned rows
// sorted longest first).  A block handles one slice of 32 systems of every
// tile assigned to it: lanes per row LPR = 32 / NB, NB systems per lane (the NB
// b-values of one direction, sharing the direction operator), NB rows per
// warp.  For every tile the block stages into a shared-memory stage:
//   - the tile's FP32 planes {A0, d0, d1, d2} (16 B per entry, contiguous per
//     tile) by one TMA bulk copy counted on the stage's mbarrier,
//   - with cp.async: the slice of p at every halo row of the tile (32 complex
//     = 256 B), MD (transformed frame), the 16-bit local column indices, and
//     the owned rows' ids, entry offsets and local indices.
// Two configurations: two stages and 512 threads, one block per SM (the next
// tile's copies overlap this tile's sums), or one stage and 256 threads, two
// blocks per SM (the blocks overlap each other).  Each staged value is read from shared memory once per nonzero that needs
// it, instead of once per nonzero from L2, and the own-row p of (p, q) comes
// from the same stage.  Within a warp the NB row groups read their NB chunks
// in rotated order (group g reads chunk (k + g) mod NB at step k), which keeps
// the reads free of bank conflicts.
#include "bt_kernels.cuh"

namespace bt {

namespace {

// shared memory of one stage of configuration c: halo rows (32 float2 each),
// then the entries' planes, MD, local indices, the owned rows' ids, entry
// offsets (one more), local indices (16-bit, copied in 4-byte words), and a
// 16-byte header with the tile's first entry, first owned row and owned rows
struct StageLayout {
  size_t halo, pk, md, li, row, hdr, total;
};
constexpr StageLayout stage_layout(int c) {
  const size_t U = (size_t)SLICE_CONF[c].umax, T = (size_t)SLICE_CONF[c].tmax, E = (size_t)SLICE_CONF[c].emax;
  const size_t halo = U * 32 * sizeof(float2), pk = E * sizeof(float4), md = E * sizeof(float),
               li = ((E + 8) * sizeof(uint16_t) + 15) / 16 * 16, row = ((T * 4 + (T + 1) * 4 + (T + 4) * 2) + 15) / 16 * 16;
  return StageLayout{halo, pk, md, li, row, 16, halo + pk + md + li + row + 16};
}
static_assert(stage_layout(0).total % 16 == 0 && stage_layout(2).total % 16 == 0, "stage alignment");
// a configuration's blocks must fit one SM's shared memory (228 KB, 1 KB
// reserved per block)
// (the stages are followed by 64 bytes of mbarriers and counters)
constexpr bool fits_sm(int c) {
  return (size_t)SLICE_CONF[c].blocks * ((size_t)SLICE_CONF[c].stages * stage_layout(c).total + 64 + 1024) <=
             228 * 1024 &&
         (size_t)SLICE_CONF[c].stages * stage_layout(c).total + 64 <= 227 * 1024;
}
static_assert(fits_sm(0) && fits_sm(1) && fits_sm(2) && fits_sm(3) && fits_sm(4),
              "slice configuration exceeds shared memory");

__device__ __forceinline__ void cpa16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa4(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Bulk (TMA) copies into shared memory, completed on an mbarrier that counts
// the bytes in flight.  A wait is bounded: past about two seconds the caller
// records a timeout instead of spinning on.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(sdst)),
               "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// one arrival on an mbarrier (release semantics at CTA scope)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// an arrival on the mbarrier made when every cp.async this thread issued so far
// has landed (the arrival is counted in the barrier's initial count)
__device__ __forceinline__ void cpa_mbar_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// generic-proxy accesses of this thread before async-proxy writes to the same shared memory
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// true when the phase of `parity` completed; false after the time limit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const long long t0 = clock64();
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && clock64() - t0 > 4000000000LL) return false;
  }
}

// 1 / d for a complex diagonal d = (re, im); the same arithmetic in both
// launches, so z = D^-1 r agrees bit for bit between them
__device__ __forceinline__ float2 diag_inv(float re, float im) {
  const float s = __frcp_rn(fmaf(re, re, im * im));
  return make_float2(re * s, -im * s);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// acc += a b
__device__ __forceinline__ void cmacf(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Per-lane FP32 partials (slot k of group g holds system (k + g) mod NB) are
// un-rotated into system order, summed over the NB row groups of the warp and
// added in FP64 to the partials kept by the lanes of group 0.
template <int NB, int LPR>
__device__ __forceinline__ void slice_flush(float2 (&a32)[NB][1], double2 (&a64)[NB][1], int g) {
  // exact selection by bit masks (a data-dependent register index would be
  // placed in local memory)
  float2 sys[NB][1];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int c = 0; c < 1; ++c) {
      unsigned vx = 0u, vy = 0u;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        const unsigned msk = (((b - g + NB) % NB) == k) ? 0xFFFFFFFFu : 0u;
        vx |= __float_as_uint(a32[k][c].x) & msk;
        vy |= __float_as_uint(a32[k][c].y) & msk;
      }
      sys[b][c] = make_float2(__uint_as_float(vx), __uint_as_float(vy));
    }
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int c = 0; c < 1; ++c) {
      float2 v = sys[b][c];
#pragma unroll
      for (int o = LPR; o < 32; o <<= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      }
      if (g == 0) {
        a64[b][c].x += (double)v.x;
        a64[b][c].y += (double)v.y;
      }
      a32[b][c] = make_float2(0.f, 0.f);
    }
}

}  // namespace

// One owned row of a staged tile: q_row = L_row p for the lane's NB systems
// (entries ea..eb of the stage, p from the staged halo rows xs), stored for the
// active systems, and (p_row, q_row) added to the lane's FP32 partials.
template <int NB, bool TRANSF>
__device__ __forceinline__ void slice_row(const float4* spk, const uint16_t* sli, const float* smd, const float2* xs,
                                          int row, int ea, int eb, int lo, const OpArgs& op, float2* __restrict__ q,
                                          float qx, float qy, float qz, float ca, const float (&cb)[NB],
                                          const float (&cc)[NB], const int (&off)[NB], const int (&colk)[NB],
                                          const bool (&act)[NB], float2 (&a32)[NB][1]) {
  constexpr bool CONJ = TRANSF;
  float2 P[NB], Q[NB];
#pragma unroll
  for (int kk = 0; kk < NB; ++kk) P[kk] = Q[kk] = make_float2(0.f, 0.f);
#pragma unroll 2
  for (int e = ea; e < eb; ++e) {
    const float4 v = spk[e];
    const int l = sli[e];
    const float m = fmaf(qx, v.y, fmaf(qy, v.z, qz * v.w));
    const float a0 = ca * v.x;
    float z1 = 0.f;
    if constexpr (TRANSF) z1 = smd[e];
    const float2* xr = xs + l * 32;
    const float2 m2 = make_float2(m, m);
#pragma unroll
    for (int kk = 0; kk < NB; ++kk) {
      const float2 xx = xr[off[kk]];
      float c = a0;
      if constexpr (TRANSF) c = fmaf(cb[kk], z1, c);
      P[kk] = __ffma2_rn(make_float2(c, c), xx, P[kk]);
      Q[kk] = __ffma2_rn(m2, xx, Q[kk]);
    }
  }
  const size_t erow = (size_t)row * op.Rp;
  const float2* pown = xs + lo * 32;
#pragma unroll
  for (int kk = 0; kk < NB; ++kk) {
    const float2 y = make_float2(fmaf(-cc[kk], Q[kk].y, P[kk].x), fmaf(cc[kk], Q[kk].x, P[kk].y));
    if (act[kk]) __stcs(q + erow + colk[kk], y);
    float2 pv = pown[off[kk]];
    if constexpr (CONJ) pv = conjf2(pv);
    const float wgt = act[kk] ? 1.f : 0.f;  // inactive systems add zeros
    cmacf(a32[kk][0], make_float2(wgt * pv.x, wgt * pv.y), y);
  }
}

// End of a slice SpMM block: the FP64 partials of (p, q) of its NW warps
// (kept by the group-0 lanes) summed per system into the block's slot of
// rs.part; the last block to arrive forms alpha for every system.
template <int NB, int NW>
__device__ __forceinline__ void slice_epilogue(char* smem, int tid, int warp, int g, int lp, int tt, int jc, int tb,
                                               const OpArgs& op, const SegPlan& spt, const KrylovState& ks,
                                               RedScratch rs, const double2 (&a64)[NB][1]) {
  constexpr int LPR = 32 / NB;
  // block reduction: group-0 lanes of each warp hold FP64 partials of the
  // slice's 32 systems (lane lp: systems L*NB .. L*NB+NB-1)
  double2* red = reinterpret_cast<double2*>(smem);  // [NW warps][32 systems]
  if (g == 0 && warp < NW) {
#pragma unroll
    for (int b = 0; b < NB; ++b) red[(size_t)warp * 32 + lp * NB + b] = a64[b][0];
  }
  __syncthreads();
  if (tid < 32) {
    double2 sum = make_double2(0.0, 0.0);
    for (int wp = 0; wp < NW; ++wp) {
      const double2 v = red[(size_t)wp * 32 + tid];
      sum.x += v.x;
      sum.y += v.y;
    }
    // slice system tid = lp * NB + b belongs to lane L = LPR jc + lp
    const int rloc = (tt * 32 + LPR * jc + tid / NB) * NB + tid % NB;
    if (rloc < op.R) reinterpret_cast<double2*>(rs.part)[(size_t)tb * op.Rp + rloc] = sum;
  }
  if (!last_block(rs.counter, gridDim.x)) return;
  if (threadIdx.x == 0 && ks.sys_iter) atomicAdd(ks.sys_iter, (unsigned long long)*ks.n_active);
  __syncthreads();
  reduce_systems<1>(rs.part, spt, op.R, op.Rp, [](int) { return false; }, [&](int s, const double2 (&t)[1]) {
    count_segment_iter(ks, s, op.R);
    krylov_alpha(ks, s, t[0]);
    ks.pend[s] = ks.active[s];  // the x update of this iteration is still to do
  });
}

// the stages, then the mbarriers and counters (64 bytes)
size_t slice_smem_bytes(int c) { return (size_t)SLICE_CONF[c].stages * stage_layout(c).total + 64; }

// ---------------------------------------------------------------- SpMM + (p, q)
// Two stages: the next tile's copies overlap this tile's sums; one stage:
// each block copies then sums, and the blocks resident on an SM overlap each
// other.  CONJ = TRANSF: CG (conjugated forms) in the transformed frame,
// COCG in the lab frame.
template <int NB, bool TRANSF, int CFG>
__global__ void __launch_bounds__(SLICE_CONF[CFG].threads, SLICE_CONF[CFG].blocks)
    k_spmm_slice(OpArgs op, HaloArgs h, SegPlan spt, int S, const float2* __restrict__ p, float2* __restrict__ q,
                 KrylovState ks, RedScratch rs) {
  if (*ks.n_active == 0) return;
  constexpr bool CONJ = TRANSF;
  constexpr int STAGES = SLICE_CONF[CFG].stages;
  constexpr int SL_UMAX = SLICE_CONF[CFG].umax, SL_TMAX = SLICE_CONF[CFG].tmax;
  constexpr StageLayout LY = stage_layout(CFG);
  constexpr size_t SL_HALO_BYTES = LY.halo, SL_PK_BYTES = LY.pk, SL_MD_BYTES = LY.md, SL_LI_BYTES = LY.li,
                   SL_STAGE_BYTES = LY.total;
  constexpr int LPR = 32 / NB;   // lanes per row
  constexpr int NT = SLICE_CONF[CFG].threads, NW = NT / 32;
  constexpr int SLOTS = NW * NB;  // rows in flight per block
  constexpr int PPC = 16 / NB;                     // 16-byte pieces per chunk of LPR complex values
  constexpr int HPT = SL_UMAX * 16 / NT;          // halo pieces per thread at most
  static_assert(SL_UMAX * 16 % NT == 0, "halo pieces per thread");
  extern __shared__ float4 sl_smem_[];
  char* smem = reinterpret_cast<char*>(sl_smem_);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int slice = blockIdx.x % S, tb = blockIdx.x / S;
  const int tt = slice / NB, jc = slice % NB;
  const int g = lane / LPR, lp = lane % LPR;
  const int L = LPR * jc + lp;
  const int r0 = (tt * 32 + L) * NB;       // first system of this lane (in its segment)
  const int c0 = tt * 32 * NB + L;         // its first column
  const int cs = tt * 32 * NB + LPR * jc;  // first column of chunk 0 of the slice
  const bool on = r0 < op.R;
  const int sg = spt.blk_seg[tb], sk = tb - spt.blk0[sg], snb = spt.blk0[sg + 1] - spt.blk0[sg];
  const OpCoef cf = op_coef(op, sg);
  const int base = sg * op.R;
  const int dsys = base + (on ? r0 : 0);
  const float qx = (float)op.qhat[3 * dsys], qy = (float)op.qhat[3 * dsys + 1], qz = (float)op.qhat[3 * dsys + 2];
  const float ca = (float)cf.a;
  // slot k holds system b = (k + g) mod NB
  float cb[NB], cc[NB];
  int off[NB], colk[NB];
  bool act[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int b = (k + g) % NB, rr = r0 + b;
    const double qq = (on && rr < op.R) ? op.q[base + rr] : 0.0;
    cb[k] = (float)(cf.bq2 * qq * qq);
    cc[k] = (float)(cf.cq * qq);
    act[k] = on && rr < op.R && ks.active[base + rr] != 0;
    off[k] = b * LPR;
    colk[k] = c0 + 32 * b;
  }
  // (p, q) per slot: FP32 over a few tiles, then warp-reduced into FP64
  float2 a32[NB][1];
  double2 a64[NB][1];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    a32[k][0] = make_float2(0.f, 0.f);
    a64[k][0] = make_double2(0.0, 0.0);
  }

  const int T0 = h.seg_tile0[sg], T1 = h.seg_tile0[sg + 1];
  auto stage_ptr = [&](int st) { return smem + (size_t)st * SL_STAGE_BYTES; };
  // one mbarrier per stage (after the stages), its phase parity in bit st
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)STAGES * SL_STAGE_BYTES);
  unsigned phase = 0u;
  // halo row ids of the 16-byte pieces this thread copies for tile tau
  // (loaded one tile ahead of their copies, so their latency overlaps the
  // sums); piece tid & 15 of halo rows (tid >> 4) + (NT / 16) j.  The tile's
  // extents come with them (m_*), and the halo range of the tile after it is
  // fetched at the same time (pre_*), so no load here waits on another.
  uint32_t rid[HPT];
  int pre_u0 = 0, pre_nu = 0, m_nu = 0, m_e0 = 0, m_ne = 0, m_R0 = 0, m_nown = 0;
  auto load_rid = [&](int tau, bool first) {
    if (first) {
      pre_u0 = __ldg(h.u0 + tau);
      pre_nu = __ldg(h.u0 + tau + 1) - pre_u0;
    }
    const int u0 = pre_u0, nu = pre_nu;
#pragma unroll
    for (int j = 0; j < HPT; ++j) {
      const int u = (tid >> 4) + (NT / 16) * j;
      rid[j] = u < nu ? (__ldg(h.ucol + u0 + u) & 0x7FFFFFFFu) : 0xFFFFFFFFu;
    }
    m_nu = nu;
    m_e0 = __ldg(h.e0 + tau);
    m_ne = __ldg(h.e0 + tau + 1) - m_e0;
    m_R0 = __ldg(h.t_r0 + tau);
    m_nown = __ldg(h.t_r0 + tau + 1) - m_R0;
    if (tau + snb < T1) {
      pre_u0 = __ldg(h.u0 + tau + snb);
      pre_nu = __ldg(h.u0 + tau + snb + 1) - pre_u0;
    }
  };
  auto issue = [&](int tau, int st) {
    char* b0 = stage_ptr(st);
    float2* sh = reinterpret_cast<float2*>(b0);
    float4* spk = reinterpret_cast<float4*>(b0 + SL_HALO_BYTES);
    float* smd = reinterpret_cast<float*>(b0 + SL_HALO_BYTES + SL_PK_BYTES);
    uint32_t* sli = reinterpret_cast<uint32_t*>(b0 + SL_HALO_BYTES + SL_PK_BYTES + SL_MD_BYTES);
    int32_t* srow = reinterpret_cast<int32_t*>(b0 + SL_HALO_BYTES + SL_PK_BYTES + SL_MD_BYTES + SL_LI_BYTES);
    int32_t* srowe = srow + SL_TMAX;
    uint32_t* srowl = reinterpret_cast<uint32_t*>(srowe + SL_TMAX + 1);
    // extents of tile tau, from load_rid(tau): nu <= SL_UMAX, ne <= the emax
    // of CFG, nown <= SL_TMAX (tile builder)
    const int nu = m_nu, e0 = m_e0, ne = m_ne, R0 = m_R0, nown = m_nown;
    if (tid == 0) *reinterpret_cast<int4*>(b0 + SL_STAGE_BYTES - 16) = make_int4(e0, R0, nown, ne);
    // the tile's planes: one bulk (TMA) copy of 16 ne contiguous bytes,
    // counted on the stage's mbarrier (issued by the thread that arms it)
    uint64_t* bar = bars + st;
    if (tid == 0) {
      fence_async_smem();
      mbar_expect(bar, (unsigned)ne * 16u);
      if (ne > 0) bulk_g2s(spk, h.pkt + e0, (unsigned)ne * 16u, bar);
    }
    // halo rows (rid: loaded by load_rid(tau)): 16-byte asynchronous copies,
    // many in flight per thread
    const int pc = tid & 15, b = pc / PPC, pp = pc - b * PPC;
#pragma unroll
    for (int j = 0; j < HPT; ++j) {
      const int u = (tid >> 4) + (NT / 16) * j;
      if (u < nu) cpa16(sh + u * 32 + b * LPR + 2 * pp, p + (size_t)rid[j] * op.Rp + cs + 32 * b + 2 * pp);
    }
    if constexpr (TRANSF)
      for (int e = tid; e < ne; e += NT) cpa4(smd + e, h.mdt + e0 + e);
    const int w0 = e0 >> 1, nw = ((e0 + ne + 1) >> 1) - w0;  // the index array is padded
    for (int w = tid; w < nw; w += NT) cpa4(sli + w, reinterpret_cast<const uint32_t*>(h.lidx) + w0 + w);
    // owned rows: ids, entry offsets, local indices
    for (int k = tid; k <= nown; k += NT) {
      if (k < nown) cpa4(srow + k, h.rows + R0 + k);
      cpa4(srowe + k, h.rowe + R0 + k);
    }
    const int l0 = R0 >> 1, nl = ((R0 + nown + 1) >> 1) - l0;  // the local-index array is padded
    for (int k = tid; k < nl; k += NT) cpa4(srowl + k, reinterpret_cast<const uint32_t*>(h.rowl) + l0 + k);
  };

  bool any = false;
#pragma unroll
  for (int k = 0; k < NB; ++k) any |= act[k];
  int ntile = 0;
  if (tid == 0) {
    for (int st = 0; st < STAGES; ++st) mbar_init(bars + st, 1u);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (__syncthreads_or(any)) {
    int tau = T0 + sk;
    if (tau < T1) load_rid(tau, true);
    if constexpr (STAGES == 2) {
      if (tau < T1) issue(tau, 0);
      cpa_commit();
      if (tau + snb < T1) load_rid(tau + snb, false);
    }
    for (int it = 0; tau < T1; tau += snb, ++it) {
      const int st = STAGES == 2 ? (it & 1) : 0;
      if constexpr (STAGES == 2) {
        if (tau + snb < T1) issue(tau + snb, st ^ 1);
        cpa_commit();
        if (tau + 2 * snb < T1) load_rid(tau + 2 * snb, false);
        cpa_wait<1>();  // this thread's copies of tile tau have landed
      } else {
        issue(tau, 0);
        cpa_commit();
        if (tau + snb < T1) load_rid(tau + snb, false);
        cpa_wait<0>();
      }
      // the stage's bulk copies (bounded wait; a timeout ends the block's work)
      const bool arrived = mbar_wait(bars + st, (phase >> st) & 1u);
      phase ^= 1u << st;
      if (__syncthreads_or(!arrived)) {
#pragma unroll
        for (int kk = 0; kk < NB; ++kk)
          if (act[kk]) ks.status[base + r0 + (kk + g) % NB] = BT_ETIMEOUT;
        // let copies still in flight land before the block's shared memory is released
        mbar_wait(bars + st, (phase >> st) & 1u ^ 1u);
        if constexpr (STAGES == 2) mbar_wait(bars + (st ^ 1), (phase >> (st ^ 1)) & 1u);
        break;
      }
      const char* b0 = stage_ptr(st);
      const float2* sh = reinterpret_cast<const float2*>(b0);
      const float4* spk = reinterpret_cast<const float4*>(b0 + SL_HALO_BYTES);
      const float* smd = reinterpret_cast<const float*>(b0 + SL_HALO_BYTES + SL_PK_BYTES);
      const int4 hdr = *reinterpret_cast<const int4*>(b0 + SL_STAGE_BYTES - 16);  // written by issue()
      const int e0 = hdr.x;
      const uint16_t* sli =
          reinterpret_cast<const uint16_t*>(b0 + SL_HALO_BYTES + SL_PK_BYTES + SL_MD_BYTES) + (e0 & 1);
      const int32_t* srow =
          reinterpret_cast<const int32_t*>(b0 + SL_HALO_BYTES + SL_PK_BYTES + SL_MD_BYTES + SL_LI_BYTES);
      const int32_t* srowe = srow + SL_TMAX;
      const int R0 = hdr.y, nown = hdr.z;
      const uint16_t* srowl = reinterpret_cast<const uint16_t*>(srowe + SL_TMAX + 1) + (R0 & 1);
      const float2* xs = sh + lp;
      for (int k = warp * NB + g; k < nown; k += SLOTS) {
        const int row = srow[k];
        const int ea = srowe[k] - e0, eb = srowe[k + 1] - e0;
        const int lo = srowl[k];
        slice_row<NB, TRANSF>(spk, sli, smd, xs, row, ea, eb, lo, op, q, qx, qy, qz, ca, cb, cc, off, colk, act,
                              a32);
      }
      if ((++ntile & 3) == 0) slice_flush<NB, LPR>(a32, a64, g);
      __syncthreads();  // the stage is refilled before it is read again
    }
    cpa_wait<0>();
  }
  slice_flush<NB, LPR>(a32, a64, g);
  __syncthreads();
  slice_epilogue<NB, NW>(smem, tid, warp, g, lp, tt, jc, tb, op, spt, ks, rs, a64);
}

// ---------------------------------------------------------------- warp-specialized SpMM
// A configuration with ws = 1: warps 0..CW-1 sum, warp CW only copies.  Each
// of the two stages has a full mbarrier (the 32 producer lanes arrive when
// their cp.async pieces have landed, and lane 0's arrival arms the planes' bulk
// copy) and an empty mbarrier (one arrival per consumer warp once the stage's
// tile has no rows left for it).  Consumer warps take NB rows at a time from
// the stage's row counter, so a warp that finishes a tile early goes on to the
// next one instead of waiting at a block barrier.  Every wait is bounded: a
// consumer that times out records BT_ETIMEOUT for its systems and raises the
// block's abort flag; the producer then stops, and before the block ends it
// waits (bounded) for every stage it filled, so no copy lands in released
// shared memory.
template <int NB, bool TRANSF, int CFG>
__global__ void __launch_bounds__(SLICE_CONF[CFG].threads, 1)
    k_spmm_slice_ws(OpArgs op, HaloArgs h, SegPlan spt, int S, const float2* __restrict__ p, float2* __restrict__ q,
                    KrylovState ks, RedScratch rs) {
  if (*ks.n_active == 0) return;
  static_assert(SLICE_CONF[CFG].ws == 1 && SLICE_CONF[CFG].stages == 2 && SLICE_CONF[CFG].umax % 32 == 0,
                "warp-specialized configuration");
  constexpr int SL_UMAX = SLICE_CONF[CFG].umax, SL_TMAX = SLICE_CONF[CFG].tmax;
  constexpr StageLayout LY = stage_layout(CFG);
  constexpr size_t SL_HALO_BYTES = LY.halo, SL_PK_BYTES = LY.pk, SL_MD_BYTES = LY.md, SL_LI_BYTES = LY.li,
                   SL_STAGE_BYTES = LY.total;
  constexpr int LPR = 32 / NB, PPC = 16 / NB;
  constexpr int CW = SLICE_CONF[CFG].threads / 32 - 1;  // consumer warps; warp CW copies
  extern __shared__ float4 sl_smem_[];
  char* smem = reinterpret_cast<char*>(sl_smem_);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int slice = blockIdx.x % S, tb = blockIdx.x / S;
  const int tt = slice / NB, jc = slice % NB;
  const int g = lane / LPR, lp = lane % LPR;
  const int L = LPR * jc + lp;
  const int r0 = (tt * 32 + L) * NB;       // first system of this lane (in its segment)
  const int c0 = tt * 32 * NB + L;         // its first column
  const int cs = tt * 32 * NB + LPR * jc;  // first column of chunk 0 of the slice
  const bool on = r0 < op.R;
  const int sg = spt.blk_seg[tb], sk = tb - spt.blk0[sg], snb = spt.blk0[sg + 1] - spt.blk0[sg];
  const OpCoef cf = op_coef(op, sg);
  const int base = sg * op.R;
  const int dsys = base + (on ? r0 : 0);
  const float qx = (float)op.qhat[3 * dsys], qy = (float)op.qhat[3 * dsys + 1], qz = (float)op.qhat[3 * dsys + 2];
  const float ca = (float)cf.a;
  float cb[NB], cc[NB];
  int off[NB], colk[NB];
  bool act[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const int b = (k + g) % NB, rr = r0 + b;
    const double qq = (on && rr < op.R) ? op.q[base + rr] : 0.0;
    cb[k] = (float)(cf.bq2 * qq * qq);
    cc[k] = (float)(cf.cq * qq);
    act[k] = on && rr < op.R && ks.active[base + rr] != 0;
    off[k] = b * LPR;
    colk[k] = c0 + 32 * b;
  }
  float2 a32[NB][1];
  double2 a64[NB][1];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    a32[k][0] = make_float2(0.f, 0.f);
    a64[k][0] = make_double2(0.0, 0.0);
  }
  const int T0 = h.seg_tile0[sg], T1 = h.seg_tile0[sg + 1];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * SL_STAGE_BYTES);
  uint64_t* empty = full + 2;
  int* cnt = reinterpret_cast<int*>(empty + 2);  // row counters of the two stages
  volatile int* abort_flag = cnt + 2;
  bool any = false;
#pragma unroll
  for (int k = 0; k < NB; ++k) any |= act[k];
  if (tid == 0) {
    mbar_init(full, 33u);
    mbar_init(full + 1, 33u);
    mbar_init(empty, (unsigned)CW);
    mbar_init(empty + 1, (unsigned)CW);
    cnt[0] = cnt[1] = 0;
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (__syncthreads_or(any)) {
    if (warp == CW) {
      // ---- producer: fill stage it & 1 with tile tau once its previous tile is consumed
      int last0 = -1, last1 = -1;  // last use of each stage
      int it = 0;
      for (int tau = T0 + sk; tau < T1; tau += snb, ++it) {
        const int st = it & 1, use = it >> 1;
        if (use > 0 && !mbar_wait(empty + st, (unsigned)(use - 1) & 1u)) break;
        if (*abort_flag) break;
        char* b0 = smem + (size_t)st * SL_STAGE_BYTES;
        float2* sh = reinterpret_cast<float2*>(b0);
        float4* spk = reinterpret_cast<float4*>(b0 + SL_HALO_BYTES);
        float* smd = reinterpret_cast<float*>(b0 + SL_HALO_BYTES + SL_PK_BYTES);
        uint32_t* sli = reinterpret_cast<uint32_t*>(b0 + SL_HALO_BYTES + SL_PK_BYTES + SL_MD_BYTES);
        int32_t* srow = reinterpret_cast<int32_t*>(b0 + SL_HALO_BYTES + SL_PK_BYTES + SL_MD_BYTES + SL_LI_BYTES);
        int32_t* srowe = srow + SL_TMAX;
        uint32_t* srowl = reinterpret_cast<uint32_t*>(srowe + SL_TMAX + 1);
        // extents (tile builder: nu <= SL_UMAX, ne <= emax, nown <= SL_TMAX)
        const int u0 = __ldg(h.u0 + tau), nu = __ldg(h.u0 + tau + 1) - u0;
        const int e0 = __ldg(h.e0 + tau), ne = __ldg(h.e0 + tau + 1) - e0;
        const int R0 = __ldg(h.t_r0 + tau), nown = __ldg(h.t_r0 + tau + 1) - R0;
        // halo row ids, 32 rows per load: lane i holds row 32 j + i
        uint32_t rid[SL_UMAX / 32];
#pragma unroll
        for (int j = 0; j < SL_UMAX / 32; ++j) {
          const int u = 32 * j + lane;
          rid[j] = u < nu ? (__ldg(h.ucol + u0 + u) & 0x7FFFFFFFu) : 0u;
        }
        if (lane == 0) {
          *reinterpret_cast<int4*>(b0 + SL_STAGE_BYTES - 16) = make_int4(e0, R0, nown, ne);
          cnt[st] = 0;
          fence_async_smem();
          mbar_expect(full + st, (unsigned)ne * 16u);  // arrival 33: arms the planes' bulk copy
          if (ne > 0) bulk_g2s(spk, h.pkt + e0, (unsigned)ne * 16u, full + st);
        }
        // halo rows: 16 lanes per row (piece lane & 15), two rows per instruction
        const int pc = lane & 15, b = pc / PPC, pp = pc - b * PPC;
#pragma unroll
        for (int j = 0; j < SL_UMAX / 32; ++j) {
#pragma unroll
          for (int v = 0; v < 16; ++v) {
            const int u = 32 * j + 2 * v + (lane >> 4);
            const uint32_t r = __shfl_sync(0xffffffffu, rid[j], 2 * v + (lane >> 4));
            if (u < nu) cpa16(sh + u * 32 + b * LPR + 2 * pp, p + (size_t)r * op.Rp + cs + 32 * b + 2 * pp);
          }
        }
        if constexpr (TRANSF)
          for (int e = lane; e < ne; e += 32) cpa4(smd + e, h.mdt + e0 + e);
        const int w0 = e0 >> 1, nw = ((e0 + ne + 1) >> 1) - w0;  // the index array is padded
        for (int w = lane; w < nw; w += 32) cpa4(sli + w, reinterpret_cast<const uint32_t*>(h.lidx) + w0 + w);
        for (int k = lane; k <= nown; k += 32) {
          if (k < nown) cpa4(srow + k, h.rows + R0 + k);
          cpa4(srowe + k, h.rowe + R0 + k);
        }
        const int l0 = R0 >> 1, nl = ((R0 + nown + 1) >> 1) - l0;  // the local-index array is padded
        for (int k = lane; k < nl; k += 32) cpa4(srowl + k, reinterpret_cast<const uint32_t*>(h.rowl) + l0 + k);
        cpa_mbar_arrive(full + st);  // arrivals 1..32: each lane's pieces have landed
        if (st == 0) last0 = use;
        else last1 = use;
      }
      // the stages this warp filled land before the block's shared memory is released
      if (last0 >= 0) mbar_wait(full, (unsigned)last0 & 1u);
      if (last1 >= 0) mbar_wait(full + 1, (unsigned)last1 & 1u);
    } else {
      // ---- consumers: rows of stage it & 1, NB at a time, until the tile has none left
      int it = 0, ntile = 0;
      for (int tau = T0 + sk; tau < T1; tau += snb, ++it) {
        const int st = it & 1, use = it >> 1;
        const bool arrived = mbar_wait(full + st, (unsigned)use & 1u);
        if (!arrived) {
#pragma unroll
          for (int kk = 0; kk < NB; ++kk)
            if (act[kk]) ks.status[base + r0 + (kk + g) % NB] = BT_ETIMEOUT;
          *abort_flag = 1;
        }
        if (!arrived || *abort_flag) break;
        const char* b0 = smem + (size_t)st * SL_STAGE_BYTES;
        const float2* sh = reinterpret_cast<const float2*>(b0);
        const float4* spk = reinterpret_cast<const float4*>(b0 + SL_HALO_BYTES);
        const float* smd = reinterpret_cast<const float*>(b0 + SL_HALO_BYTES + SL_PK_BYTES);
        const int4 hdr = *reinterpret_cast<const int4*>(b0 + SL_STAGE_BYTES - 16);  // written by the producer
        const int e0 = hdr.x, R0 = hdr.y, nown = hdr.z;
        const uint16_t* sli =
            reinterpret_cast<const uint16_t*>(b0 + SL_HALO_BYTES + SL_PK_BYTES + SL_MD_BYTES) + (e0 & 1);
        const int32_t* srow =
            reinterpret_cast<const int32_t*>(b0 + SL_HALO_BYTES + SL_PK_BYTES + SL_MD_BYTES + SL_LI_BYTES);
        const int32_t* srowe = srow + SL_TMAX;
        const uint16_t* srowl = reinterpret_cast<const uint16_t*>(srowe + SL_TMAX + 1) + (R0 & 1);
        const float2* xs = sh + lp;
        for (;;) {
          int k0 = 0;
          if (lane == 0) k0 = atomicAdd(cnt + st, NB);
          k0 = __shfl_sync(0xffffffffu, k0, 0);
          if (k0 >= nown) break;
          const int k = k0 + g;  // one row per row group of the warp
          if (k < nown) {
            const int row = srow[k];
            const int ea = srowe[k] - e0, eb = srowe[k + 1] - e0;
            const int lo = srowl[k];
            slice_row<NB, TRANSF>(spk, sli, smd, xs, row, ea, eb, lo, op, q, qx, qy, qz, ca, cb, cc, off, colk, act,
                                  a32);
          }
        }
        if ((++ntile & 3) == 0) slice_flush<NB, LPR>(a32, a64, g);
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + st);  // this warp is done with the stage
      }
    }
  }
  slice_flush<NB, LPR>(a32, a64, g);
  __syncthreads();
  slice_epilogue<NB, CW>(smem, tid, warp, g, lp, tt, jc, tb, op, spt, ks, rs, a64);
}

// ---------------------------------------------------------------- vector updates
// Column map of the two elementwise launches: each thread owns two adjacent
// columns (16-byte accesses) and, inside the block's contiguous share of its
// segment's rows, every rpp-th row.
struct PairMap {
  int TPR, rpp, cp, ro, nch;
  bool live;
  __device__ PairMap(int Rp) {
    const int half = Rp / 2;  // column pairs per row
    TPR = half < 256 ? half : 256;
    rpp = 256 / TPR;
    cp = threadIdx.x % TPR;
    ro = threadIdx.x / TPR;
    nch = (half + 255) / 256;
    live = (int)threadIdx.x < rpp * TPR;
  }
};

// per-system constants of the Jacobi diagonal d = A0_ii + b MD_ii + i c (qhat . Pd_ii)
struct DiagCoef {
  float cb, cc, qx, qy, qz;
};
__device__ __forceinline__ DiagCoef diag_coef(const OpArgs& op, const OpCoef& cf, int s, bool valid) {
  const double qq = valid ? op.q[s] : 0.0;
  DiagCoef d;
  d.cb = (float)(cf.bq2 * qq * qq);
  d.cc = (float)(cf.cq * qq);
  d.qx = valid ? (float)op.qhat[3 * s] : 0.f;
  d.qy = valid ? (float)op.qhat[3 * s + 1] : 0.f;
  d.qz = valid ? (float)op.qhat[3 * s + 2] : 0.f;
  return d;
}
__device__ __forceinline__ float2 diag_of(const DiagCoef& c, float4 dg, float dm) {
  return make_float2(fmaf(c.cb, dm, dg.x), c.cc * fmaf(c.qx, dg.y, fmaf(c.qy, dg.z, c.qz * dg.w)));
}

// r -= alpha q; z = D^-1 r; rho' = (r, z), |r|^2 (FP32 over at most 32 rows,
// then FP64); the last block applies the convergence tests and forms beta.
template <bool CONJ>
__global__ void __launch_bounds__(256, 2) k_slice_r(OpArgs op, VecArgs va, float2* __restrict__ r,
                                                    const float2* __restrict__ q, KrylovState ks, RedScratch rs) {
  if (*ks.n_active == 0) return;
  constexpr int U = 4;  // rows in flight per thread
  const int Rp = va.Rp;
  const PairMap pm(Rp);
  BT_SEG_BEGIN(va.sp);
  const int64_t per = (sr1_ - sr0_ + snb_ - 1) / snb_;
  const int64_t rb = sr0_ + (int64_t)sk_ * per, re = min(sr1_, rb + per);
  const OpCoef cf = op_coef(op, sg_);
  const int base = sg_ * va.R;
  __shared__ double2 sred[256][2][2];
  for (int ch = 0; ch < pm.nch; ++ch) {
    const int col = 2 * (pm.cp + 256 * ch);
    double2 acc[2][2] = {{make_double2(0, 0), make_double2(0, 0)}, {make_double2(0, 0), make_double2(0, 0)}};
    bool ac[2] = {false, false};
    float2 al[2];
    DiagCoef dc[2];
    if (pm.live && col < Rp) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int rl = sys_of_col(col + u, va.nb), s = base + rl;
        ac[u] = rl < va.R && ks.active[s] != 0;
        al[u] = ac[u] ? make_float2((float)ks.alpha[2 * s], (float)ks.alpha[2 * s + 1]) : make_float2(0.f, 0.f);
        dc[u] = diag_coef(op, cf, s, rl < va.R);
      }
    }
    if (ac[0] || ac[1]) {
      float2 fr[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      float fn[2] = {0.f, 0.f};
      int cnt = 0;
      for (int64_t i0 = rb + pm.ro; i0 < re; i0 += U * pm.rpp) {
        float4 rv[U], qv[U], dg[U];
        float dm[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t i = i0 + (int64_t)k * pm.rpp;
          if (i < re) {
            const size_t e = (size_t)i * Rp + col;
            rv[k] = *reinterpret_cast<const float4*>(r + e);
            qv[k] = __ldcs(reinterpret_cast<const float4*>(q + e));
            dg[k] = __ldg(va.diag32 + i);
            dm[k] = op.transformed ? __ldg(va.diag_md32 + i) : 0.f;
          }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t i = i0 + (int64_t)k * pm.rpp;
          if (i >= re) break;
          float2 rs2[2] = {make_float2(rv[k].x, rv[k].y), make_float2(rv[k].z, rv[k].w)};
          const float2 qs[2] = {make_float2(qv[k].x, qv[k].y), make_float2(qv[k].z, qv[k].w)};
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (!ac[u]) continue;
            cmacf(rs2[u], make_float2(-al[u].x, -al[u].y), qs[u]);
            const float2 d = diag_of(dc[u], dg[k], dm[k]);
            const float2 z = cmulf(rs2[u], diag_inv(d.x, d.y));
            cmacf(fr[u], CONJ ? conjf2(rs2[u]) : rs2[u], z);
            fn[u] = fmaf(rs2[u].x, rs2[u].x, fmaf(rs2[u].y, rs2[u].y, fn[u]));
          }
          *reinterpret_cast<float4*>(r + (size_t)i * Rp + col) = make_float4(rs2[0].x, rs2[0].y, rs2[1].x, rs2[1].y);
        }
        if (++cnt == 8) {  // FP32 over at most 32 rows, then FP64
          cnt = 0;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            acc[u][0].x += fr[u].x;
            acc[u][0].y += fr[u].y;
            acc[u][1].x += fn[u];
            fr[u] = make_float2(0.f, 0.f);
            fn[u] = 0.f;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        acc[u][0].x += fr[u].x;
        acc[u][0].y += fr[u].y;
        acc[u][1].x += fn[u];
      }
    }
    // block reduction over the rows-per-pass groups; partials [block][system][2]
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      sred[threadIdx.x][u][0] = acc[u][0];
      sred[threadIdx.x][u][1] = acc[u][1];
    }
    __syncthreads();
    if ((int)threadIdx.x < pm.TPR && col < Rp) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        double2 s0 = make_double2(0, 0), s1 = make_double2(0, 0);
        for (int o = 0; o < pm.rpp; ++o) {
          const double2 a0 = sred[o * pm.TPR + threadIdx.x][u][0], a1 = sred[o * pm.TPR + threadIdx.x][u][1];
          s0.x += a0.x;
          s0.y += a0.y;
          s1.x += a1.x;
        }
        const int rl = sys_of_col(col + u, va.nb);
        if (rl < va.R) {
          double2* o2 = reinterpret_cast<double2*>(rs.part) + ((size_t)blockIdx.x * Rp + rl) * 2;
          o2[0] = s0;
          o2[1] = s1;
        }
      }
    }
    __syncthreads();
  }
  if (!last_block(rs.counter, gridDim.x)) return;
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  reduce_systems<2>(rs.part, va.sp, va.R, Rp, [&](int s) { return !ks.active[s]; },
                    [&](int s, const double2 (&o)[2]) {
                      if (krylov_step_finish(ks, s, o, nullptr)) atomicAdd(&s_cnt, 1);
                    });
  __syncthreads();
  if (threadIdx.x == 0) *ks.n_active = s_cnt;
}

// x += alpha p for the systems of the last SpMM (pend), and p = D^-1 r + beta p
// for those still active; the last block clears pend, so a launch after the
// loop has ended changes nothing.
__global__ void __launch_bounds__(256, 2) k_slice_xp(OpArgs op, VecArgs va, float2* __restrict__ x,
                                                     float2* __restrict__ p, const float2* __restrict__ r,
                                                     KrylovState ks, RedScratch rs) {
  constexpr int U = 4;  // rows in flight per thread
  const int Rp = va.Rp;
  const PairMap pm(Rp);
  BT_SEG_BEGIN(va.sp);
  const int64_t per = (sr1_ - sr0_ + snb_ - 1) / snb_;
  const int64_t rb = sr0_ + (int64_t)sk_ * per, re = min(sr1_, rb + per);
  const OpCoef cf = op_coef(op, sg_);
  const int base = sg_ * va.R;
  if (pm.live) {
    for (int ch = 0; ch < pm.nch; ++ch) {
      const int col = 2 * (pm.cp + 256 * ch);
      if (col >= Rp) continue;
      bool pd[2], ac[2];
      float2 al[2], be[2];
      DiagCoef dc[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int rl = sys_of_col(col + u, va.nb), s = base + rl;
        pd[u] = rl < va.R && ks.pend[s] != 0;
        ac[u] = pd[u] && ks.active[s] != 0;
        al[u] = pd[u] ? make_float2((float)ks.alpha[2 * s], (float)ks.alpha[2 * s + 1]) : make_float2(0.f, 0.f);
        be[u] = ac[u] ? make_float2((float)ks.beta[2 * s], (float)ks.beta[2 * s + 1]) : make_float2(0.f, 0.f);
        dc[u] = diag_coef(op, cf, s, rl < va.R);
      }
      if (!pd[0] && !pd[1]) continue;
      const bool anyp = ac[0] || ac[1];
      for (int64_t i0 = rb + pm.ro; i0 < re; i0 += U * pm.rpp) {
        float4 xv[U], pv[U], rv[U], dg[U];
        float dm[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t i = i0 + (int64_t)k * pm.rpp;
          if (i < re) {
            const size_t e = (size_t)i * Rp + col;
            xv[k] = *reinterpret_cast<const float4*>(x + e);
            pv[k] = *reinterpret_cast<const float4*>(p + e);
            if (anyp) {
              rv[k] = __ldcs(reinterpret_cast<const float4*>(r + e));
              dg[k] = __ldg(va.diag32 + i);
              dm[k] = op.transformed ? __ldg(va.diag_md32 + i) : 0.f;
            }
          }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t i = i0 + (int64_t)k * pm.rpp;
          if (i >= re) break;
          float2 xs[2] = {make_float2(xv[k].x, xv[k].y), make_float2(xv[k].z, xv[k].w)};
          float2 ps[2] = {make_float2(pv[k].x, pv[k].y), make_float2(pv[k].z, pv[k].w)};
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (!pd[u]) continue;
            cmacf(xs[u], al[u], ps[u]);
            if (ac[u]) {
              const float2 rr = u == 0 ? make_float2(rv[k].x, rv[k].y) : make_float2(rv[k].z, rv[k].w);
              const float2 d = diag_of(dc[u], dg[k], dm[k]);
              float2 np = cmulf(rr, diag_inv(d.x, d.y));
              cmacf(np, be[u], ps[u]);
              ps[u] = np;
            }
          }
          const size_t e = (size_t)i * Rp + col;
          *reinterpret_cast<float4*>(x + e) = make_float4(xs[0].x, xs[0].y, xs[1].x, xs[1].y);
          if (anyp) *reinterpret_cast<float4*>(p + e) = make_float4(ps[0].x, ps[0].y, ps[1].x, ps[1].y);
        }
      }
    }
  }
  if (!last_block(rs.counter, gridDim.x)) return;
  for (int s = threadIdx.x; s < va.sp.G * va.R; s += blockDim.x) ks.pend[s] = 0;
}

// ---------------------------------------------------------------- start of an inner solve
// r = r_res / scale_s, z = D^-1 r, p = z, x = 0; rho = (r, z), |r|^2 (FP32 over
// at most 32 rows, then FP64).  The last block initialises the per-system
// Krylov state exactly as the row variant's initialisation does.
__device__ __forceinline__ double2 load_res_d(const double2* p, size_t e) { return p[e]; }
__device__ __forceinline__ double2 load_res_d(const float4* p, size_t e) {
  const float4 v = __ldcs(p + e);
  return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}
template <class TR, bool CONJ>
__global__ void __launch_bounds__(256, 2) k_slice_init(OpArgs op, VecArgs va, const TR* __restrict__ rres,
                                                       const double* __restrict__ scale,
                                                       const int* __restrict__ ref_active, float2* __restrict__ x,
                                                       float2* __restrict__ r, float2* __restrict__ p, KrylovState ks,
                                                       double tol, RedScratch rs) {
  constexpr int U = 4;  // rows in flight per thread
  const int Rp = va.Rp;
  const PairMap pm(Rp);
  BT_SEG_BEGIN(va.sp);
  const int64_t per = (sr1_ - sr0_ + snb_ - 1) / snb_;
  const int64_t rb = sr0_ + (int64_t)sk_ * per, re = min(sr1_, rb + per);
  const OpCoef cf = op_coef(op, sg_);
  const int base = sg_ * va.R;
  __shared__ double2 sred[256][2][2];
  for (int ch = 0; ch < pm.nch; ++ch) {
    const int col = 2 * (pm.cp + 256 * ch);
    double2 acc[2][2] = {{make_double2(0, 0), make_double2(0, 0)}, {make_double2(0, 0), make_double2(0, 0)}};
    if (pm.live && col < Rp) {
      bool ac[2];
      double inv[2];
      DiagCoef dc[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int rl = sys_of_col(col + u, va.nb), s = base + rl;
        ac[u] = rl < va.R && ref_active[s] != 0;
        inv[u] = (scale && ac[u] && scale[s] > 0) ? 1.0 / scale[s] : 1.0;
        dc[u] = diag_coef(op, cf, s, rl < va.R);
      }
      float2 fr[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      float fn[2] = {0.f, 0.f};
      int cnt = 0;
      for (int64_t i0 = rb + pm.ro; i0 < re; i0 += U * pm.rpp) {
        double2 v[U][2];
        float4 dg[U];
        float dm[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t i = i0 + (int64_t)k * pm.rpp;
          if (i < re) {
            const size_t e = (size_t)i * Rp + col;
#pragma unroll
            for (int u = 0; u < 2; ++u) v[k][u] = ac[u] ? load_res_d(rres, e + u) : make_double2(0, 0);
            dg[k] = __ldg(va.diag32 + i);
            dm[k] = op.transformed ? __ldg(va.diag_md32 + i) : 0.f;
          }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t i = i0 + (int64_t)k * pm.rpp;
          if (i >= re) break;
          float2 rv[2], zv[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            rv[u] = make_float2((float)(v[k][u].x * inv[u]), (float)(v[k][u].y * inv[u]));
            const float2 d = diag_of(dc[u], dg[k], dm[k]);
            zv[u] = cmulf(rv[u], diag_inv(d.x, d.y));
            cmacf(fr[u], CONJ ? conjf2(rv[u]) : rv[u], zv[u]);
            fn[u] = fmaf(rv[u].x, rv[u].x, fmaf(rv[u].y, rv[u].y, fn[u]));
          }
          const size_t e = (size_t)i * Rp + col;
          *reinterpret_cast<float4*>(r + e) = make_float4(rv[0].x, rv[0].y, rv[1].x, rv[1].y);
          *reinterpret_cast<float4*>(p + e) = make_float4(zv[0].x, zv[0].y, zv[1].x, zv[1].y);
          *reinterpret_cast<float4*>(x + e) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (++cnt == 8) {  // FP32 over at most 32 rows, then FP64
          cnt = 0;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            acc[u][0].x += fr[u].x;
            acc[u][0].y += fr[u].y;
            acc[u][1].x += fn[u];
            fr[u] = make_float2(0.f, 0.f);
            fn[u] = 0.f;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        acc[u][0].x += fr[u].x;
        acc[u][0].y += fr[u].y;
        acc[u][1].x += fn[u];
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      sred[threadIdx.x][u][0] = acc[u][0];
      sred[threadIdx.x][u][1] = acc[u][1];
    }
    __syncthreads();
    if ((int)threadIdx.x < pm.TPR && col < Rp) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        double2 s0 = make_double2(0, 0), s1 = make_double2(0, 0);
        for (int o = 0; o < pm.rpp; ++o) {
          const double2 a0 = sred[o * pm.TPR + threadIdx.x][u][0], a1 = sred[o * pm.TPR + threadIdx.x][u][1];
          s0.x += a0.x;
          s0.y += a0.y;
          s1.x += a1.x;
        }
        const int rl = sys_of_col(col + u, va.nb);
        if (rl < va.R) {
          double2* o2 = reinterpret_cast<double2*>(rs.part) + ((size_t)blockIdx.x * Rp + rl) * 2;
          o2[0] = s0;
          o2[1] = s1;
        }
      }
    }
    __syncthreads();
  }
  if (!last_block(rs.counter, gridDim.x)) return;
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  reduce_systems<2>(rs.part, va.sp, va.R, Rp, [](int) { return false; }, [&](int s, const double2 (&o)[2]) {
    ks.rho[2 * s] = o[0].x;
    ks.rho[2 * s + 1] = o[0].y;
    ks.rr0[s] = o[1].x;
    ks.rr[s] = o[1].x;
    ks.tol2[s] = tol * tol * o[1].x;
    ks.iter[s] = 0;
    ks.rr_best[s] = o[1].x;
    ks.it_best[s] = 0;
    ks.pend[s] = 0;
    int a = ref_active[s] && o[1].x > 0;
    if (ref_active[s] && !isfinite(o[1].x)) {
      a = 0;
      ks.status[s] = BT_ENAN;
    }
    ks.active[s] = a;
    if (a) atomicAdd(&s_cnt, 1);
  });
  __syncthreads();
  if (threadIdx.x == 0) *ks.n_active = s_cnt;
}

// ---------------------------------------------------------------- launchers
template <int NB, bool TRANSF>
static void slice_attr() {
  cudaFuncSetAttribute(k_spmm_slice<NB, TRANSF, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)slice_smem_bytes(0));
  cudaFuncSetAttribute(k_spmm_slice<NB, TRANSF, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)slice_smem_bytes(1));
  cudaFuncSetAttribute(k_spmm_slice<NB, TRANSF, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)slice_smem_bytes(2));
  cudaFuncSetAttribute(k_spmm_slice<NB, TRANSF, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)slice_smem_bytes(3));
  cudaFuncSetAttribute(k_spmm_slice_ws<NB, TRANSF, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)slice_smem_bytes(4));
}
void slice_prepare() {
  slice_attr<4, false>();
  slice_attr<4, true>();
  slice_attr<2, false>();
  slice_attr<2, true>();
  slice_attr<1, false>();
  slice_attr<1, true>();
}

// conj must equal op.transformed (CG in the transformed frame, COCG in the
// lab frame), as everywhere in the library
void launch_spmm_slice(const OpArgs& op, const HaloArgs& h, const SegPlan& spt, const float2* p, float2* q,
                       const KrylovState& ks, RedScratch rs, int conj, int nb, int cfg, cudaStream_t st) {
  (void)conj;
  const int S = op.Rp / 32;
  const dim3 grid(spt.nblk * S);
  const size_t sm = slice_smem_bytes(cfg);
#define BT_SL_CASE(NBV, CFGV)                                                                          \
  {                                                                                                    \
    constexpr int NT_ = SLICE_CONF[CFGV].threads;                                                      \
    if (op.transformed) k_spmm_slice<NBV, true, CFGV><<<grid, NT_, sm, st>>>(op, h, spt, S, p, q, ks, rs); \
    else k_spmm_slice<NBV, false, CFGV><<<grid, NT_, sm, st>>>(op, h, spt, S, p, q, ks, rs);            \
  }
#define BT_SL_NB(CFGV)                  \
  switch (nb) {                         \
    case 4: BT_SL_CASE(4, CFGV) break;  \
    case 2: BT_SL_CASE(2, CFGV) break;  \
    default: BT_SL_CASE(1, CFGV) break; \
  }
#define BT_SL_WS_CASE(NBV, CFGV)                                                                        \
  {                                                                                                    \
    constexpr int NT_ = SLICE_CONF[CFGV].threads;                                                      \
    if (op.transformed) k_spmm_slice_ws<NBV, true, CFGV><<<grid, NT_, sm, st>>>(op, h, spt, S, p, q, ks, rs); \
    else k_spmm_slice_ws<NBV, false, CFGV><<<grid, NT_, sm, st>>>(op, h, spt, S, p, q, ks, rs);            \
  }
  switch (cfg) {
    case 0: BT_SL_NB(0) break;
    case 1: BT_SL_NB(1) break;
    case 2: BT_SL_NB(2) break;
    case 3: BT_SL_NB(3) break;
    default:
      switch (nb) {
        case 4: BT_SL_WS_CASE(4, 4) break;
        case 2: BT_SL_WS_CASE(2, 4) break;
        default: BT_SL_WS_CASE(1, 4) break;
      }
      break;
  }
#undef BT_SL_WS_CASE
#undef BT_SL_NB
#undef BT_SL_CASE
}

void launch_slice_r(const OpArgs& op, const VecArgs& va, float2* r, const float2* q, const KrylovState& ks,
                    RedScratch rs, int conj, cudaStream_t st) {
  if (conj) k_slice_r<true><<<va.sp.nblk, 256, 0, st>>>(op, va, r, q, ks, rs);
  else k_slice_r<false><<<va.sp.nblk, 256, 0, st>>>(op, va, r, q, ks, rs);
}

void launch_slice_xp(const OpArgs& op, const VecArgs& va, float2* x, float2* p, const float2* r,
                     const KrylovState& ks, RedScratch rs, cudaStream_t st) {
  k_slice_xp<<<va.sp.nblk, 256, 0, st>>>(op, va, x, p, r, ks, rs);
}

void launch_slice_init(const OpArgs& op, const VecArgs& va, const void* rres, int df, const double* scale,
                       const int* ref_active, float2* x, float2* r, float2* p, const KrylovState& ks, double tol,
                       RedScratch rs, int conj, cudaStream_t st) {
  const int g = va.sp.nblk;
  if (df) {
    const float4* rr = static_cast<const float4*>(rres);
    if (conj) k_slice_init<float4, true><<<g, 256, 0, st>>>(op, va, rr, scale, ref_active, x, r, p, ks, tol, rs);
    else k_slice_init<float4, false><<<g, 256, 0, st>>>(op, va, rr, scale, ref_active, x, r, p, ks, tol, rs);
  } else {
    const double2* rr = static_cast<const double2*>(rres);
    if (conj) k_slice_init<double2, true><<<g, 256, 0, st>>>(op, va, rr, scale, ref_active, x, r, p, ks, tol, rs);
    else k_slice_init<double2, false><<<g, 256, 0, st>>>(op, va, rr, scale, ref_active, x, r, p, ks, tol, rs);
  }
}

}  // namespace bt
