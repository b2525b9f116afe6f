// Dense multi-target gates on complex64 state vectors on the tensor cores
// (tcgen05, sm_100-family).  A gate U on m targets maps every block of 2^m
// amplitudes v (the amplitudes that differ only in the target bits, Eq. 1
// with the pair replaced by a block) to U v.  For 128 blocks at a time this
// is one real matrix product
//     W^T = V^T B,   V^T: 128 x 2^(m+1) rows [Re v, Im v],
//     B (2^(m+1) x 2^(m+1)) = [[Re U^T, Im U^T], [-Im U^T, Re U^T]],
// so row b of the result is [Re (U v_b), Im (U v_b)].  The operands are
// FP32; the tensor cores multiply TF32 (11 significant bits), so each
// operand is split x = hi + lo with hi = x rounded to TF32 and lo = x - hi
// (exact, at most 12 significant bits, of which TF32 keeps 11), and the
// product is accumulated as lo*hi + hi*lo + hi*hi in FP32 (the dropped
// lo*lo term and the lost bit of lo are about 2^-23 relative): close to
// FP32 accuracy (measured: a few units of 1e-7 of the largest amplitude per
// gate).
//
// Two kernels.  The staged one (k_sv_multi_tcs, below) serves registers
// with at least seven qubits that are neither target nor control: tiles
// copied in address order into shared memory two tiles ahead, A written to
// tensor memory, results stored coalesced.  The register-gather one
// (k_sv_multi_tc) serves the rest and the "multi_tc_stage" 0 option: per
// CTA 128 threads, one block (GEMM row) per thread, gathered into
// registers; operands in shared memory in the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per core matrix; consecutive core
// matrices 128 bytes apart along the rows, R*16 bytes apart along K), the
// accumulator (128 lanes x 2^(m+1) FP32 columns) in tensor memory.  In
// both, one thread issues the MMAs and commits them to an mbarrier; every
// thread waits (bounded) and reads its row back with tcgen05.ld.  Here the
// next tile's gather is issued before the wait, so global loads overlap
// the MMAs and the stores.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace qs {

constexpr int kTcRows = 128;  // GEMM rows (blocks) per tile = threads per CTA

template <int MT>
struct TcParams {
  uint8_t t[8];                     // target qubits; bit k of the block index is t[k]
  // coalesced mode: a tile's 128 x 2^m amplitudes enumerated in address
  // order, bit k of the enumeration index at qubit pos[k] (the 7 lowest
  // free qubits and the targets, ascending); role[k] = 0x80 | u for target
  // t[u], else the block-index bit it carries
  uint8_t pos[16];
  uint8_t role[16];
  uint8_t split;                    // staged kernel: qubit 0 is a control (pairs copied as two 8 B halves)
  float2 u[1 << (2 * MT)];          // row-major matrix
};

// Shared-memory bytes of one CTA: A hi/lo (128 x K), B hi/lo (N x K), the
// block offsets, the coalesced mode's per-index offsets, rows and columns,
// the mbarrier and the tensor-memory address slot.
template <int MT>
__host__ __device__ constexpr size_t tc_smem_bytes() {
  return size_t(2) * kTcRows * (2 << MT) * 4 + size_t(2) * (2 << MT) * (2 << MT) * 4 +
         2 * sizeof(int64_t) * (1 << MT) + 2 * (1 << MT) + 64;
}

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (between core matrices along K), stride byte offset (between core
// matrices along M / N), all in 16-byte units; bits 46-48 = 0b001; no
// swizzle, base offset 0.
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t kstride, uint32_t rstride) {
  return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t((kstride >> 4) & 0x3FFFu) << 16) |
         (uint64_t((rstride >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor, kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase with the given parity, for at most max_ns nanoseconds
// of the global timer (each try_wait suspends for at most a short,
// system-defined time, so the deadline is checked between tries).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t max_ns = 1000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > max_ns) return false;
  }
}

// x rounded to the nearest TF32 value (ties away from zero); x - tf32_hi(x)
// is exact in FP32 and has at most 12 significant bits.
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
}

// Element (r, k) of an R-row K-major operand, in floats.
template <int R>
__device__ __forceinline__ int at(int r, int k) {
  return (k >> 2) * (R * 4) + (r >> 3) * 32 + (r & 7) * 4 + (k & 3);
}

#define QS_R32(m, r, o)                                                                              \
  m(r[o + 0]), m(r[o + 1]), m(r[o + 2]), m(r[o + 3]), m(r[o + 4]), m(r[o + 5]), m(r[o + 6]), m(r[o + 7]), \
      m(r[o + 8]), m(r[o + 9]), m(r[o + 10]), m(r[o + 11]), m(r[o + 12]), m(r[o + 13]), m(r[o + 14]),     \
      m(r[o + 15]), m(r[o + 16]), m(r[o + 17]), m(r[o + 18]), m(r[o + 19]), m(r[o + 20]), m(r[o + 21]),   \
      m(r[o + 22]), m(r[o + 23]), m(r[o + 24]), m(r[o + 25]), m(r[o + 26]), m(r[o + 27]), m(r[o + 28]),   \
      m(r[o + 29]), m(r[o + 30]), m(r[o + 31])
#define QS_OUT(x) "=r"(x)
#define QS_INOUT(x) "+r"(x)

// Columns [O, O + 32) of the accumulator, this warp's 32 lanes, into
// r[O .. O + 32).  Asynchronous: the registers hold the values only after
// wait_ld, which takes them as operands so that no use moves above it.
template <int O, int N>
__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t (&r)[N]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : QS_R32(QS_OUT, r, O)
      : "r"(taddr));
}

template <int N>
__device__ __forceinline__ void wait_ld(uint32_t (&r)[N]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : QS_R32(QS_INOUT, r, 0)::"memory");
  if constexpr (N > 32) asm volatile("" : QS_R32(QS_INOUT, r, 32));
}

// Columns [O, O + 32) of this warp's 32 lanes written from r[0 .. 32)
// (thread i: lane 32 * warp + i).  Asynchronous: complete after wait_st.
template <int N>
__device__ __forceinline__ void st32(uint32_t taddr, const uint32_t (&r)[N]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

// 16-column forms: columns [taddr, taddr + 16) of this warp's lanes into
// r[O .. O + 16) (ld16) or from r[0 .. 16) (st16).
template <int O, int N>
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&r)[N]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[O + 0]), "=r"(r[O + 1]), "=r"(r[O + 2]), "=r"(r[O + 3]), "=r"(r[O + 4]), "=r"(r[O + 5]),
        "=r"(r[O + 6]), "=r"(r[O + 7]), "=r"(r[O + 8]), "=r"(r[O + 9]), "=r"(r[O + 10]), "=r"(r[O + 11]),
        "=r"(r[O + 12]), "=r"(r[O + 13]), "=r"(r[O + 14]), "=r"(r[O + 15])
      : "r"(taddr));
}

template <int N>
__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t (&r)[N]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D (tensor memory) (+)= A (tensor memory, 128 lanes = rows, one TF32 per
// column) x B (shared-memory descriptor).
__device__ __forceinline__ void mma_tf32_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Asynchronous global -> shared copies (cp.async; this thread's groups).
__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shared-memory position (in 8-byte elements) of tile element e in the
// staged kernel: its 16-byte chunk c = e >> 1 moves to c ^ h(c >> 3), h the
// XOR of c's 3-bit groups, so that the rows a warp reads (any five of the
// enumeration bits) spread over the banks; linear over GF(2), so the
// position of a union of disjoint bit sets is the XOR of their positions.
__host__ __device__ constexpr uint32_t chunk_swz(uint32_t c) {
  return c ^ (((c >> 3) ^ (c >> 6) ^ (c >> 9)) & 7u);
}
__host__ __device__ constexpr uint32_t elem_pos(uint32_t e) { return (chunk_swz(e >> 1) << 1) | (e & 1u); }

}  // namespace tc

// status: bit 0 set when a wait for the tensor cores ran out (1 s of the
// global timer; the kernel then stops; the amplitudes of unfinished tiles
// are unchanged or partly written).
// COAL: targets among the lowest qubits, where one thread's block is a few
// contiguous runs and a warp's per-block loads would not coalesce: the CTA
// loads the tile in address order into a row-swizzled staging buffer (the
// A lo area) and each thread then reads its block from it; results go back
// the same way through the A hi area (free once the MMAs are done).
// Requires nsel >= 128 (seven free qubits).
template <int MT, bool COAL>
__global__ void __launch_bounds__(kTcRows) k_sv_multi_tc(float2* __restrict__ a, int64_t nsel, Fixed fx,
                                                        const __grid_constant__ TcParams<MT> p,
                                                        unsigned* status) {
  constexpr int D2 = 1 << MT, KD = 2 * D2, ND = 2 * D2;
  constexpr uint32_t kA = kTcRows * KD * 4, kB = ND * KD * 4;  // bytes of one A / B operand
  constexpr uint32_t kIdesc = tc::idesc_tf32(kTcRows, ND);
  extern __shared__ __align__(1024) uint8_t smem[];
  float* sAh = reinterpret_cast<float*>(smem);
  float* sAl = reinterpret_cast<float*>(smem + kA);
  float* sBh = reinterpret_cast<float*>(smem + 2 * kA);
  float* sBl = reinterpret_cast<float*>(smem + 2 * kA + kB);
  int64_t* toff = reinterpret_cast<int64_t*>(smem + 2 * kA + 2 * kB);
  int64_t* ioff = toff + D2;
  uint8_t* irow = reinterpret_cast<uint8_t*>(ioff + D2);
  uint8_t* il = irow + D2;
  constexpr uint32_t kBar = (2 * kA + 2 * kB + 18 * D2 + 7) / 8 * 8;  // after toff, ioff, irow, il
  static_assert(kBar + 16 <= tc_smem_bytes<MT>(), "shared-memory layout");
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  // coalesced mode: this thread's part (enumeration bits 0..6) of every
  // element's address (tdep), block row (trow) and column (tl)
  int64_t tdep = 0;
  int trow = 0, tl = 0;
  if constexpr (COAL) {
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      if (!((tid >> k) & 1)) continue;
      tdep += int64_t(1) << p.pos[k];
      if (p.role[k] & 0x80) tl |= 1 << (p.role[k] & 0x7F);
      else trow |= 1 << p.role[k];
    }
  }

  // B = [[Re U^T, Im U^T], [-Im U^T, Re U^T]] stored N x K (row n = output
  // column): row n < D2 gives Re w[n], row D2 + n gives Im w[n].
  for (int e = tid; e < ND * KD; e += kTcRows) {
    const int n = e / KD, k = e % KD;
    const float2 u = p.u[(n & (D2 - 1)) * D2 + (k & (D2 - 1))];
    const float v = n < D2 ? (k < D2 ? u.x : -u.y) : (k < D2 ? u.y : u.x);
    const float h = tc::tf32_hi(v);
    sBh[tc::at<ND>(n, k)] = h;
    sBl[tc::at<ND>(n, k)] = v - h;
  }
  if (tid < D2) {
    int64_t o = 0;
    for (int k = 0; k < MT; ++k)
      if ((tid >> k) & 1) o += int64_t(1) << p.t[k];
    toff[tid] = o;
    if constexpr (COAL) {  // enumeration bits 7..7+m-1 from the element index i = tid
      int64_t d = 0;
      int rw = 0, cl = 0;
      for (int k = 0; k < MT; ++k) {
        if (!((tid >> k) & 1)) continue;
        const uint8_t r = p.role[7 + k];
        d += int64_t(1) << p.pos[7 + k];
        if (r & 0x80) cl |= 1 << (r & 0x7F);
        else rw |= 1 << r;
      }
      ioff[tid] = d;
      irow[tid] = uint8_t(rw);
      il[tid] = uint8_t(cl);
    }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tslot)),
                 "r"(uint32_t(ND)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t bar_a = tc::smem_u32(bar);
  const uint32_t ah = tc::smem_u32(sAh), al = tc::smem_u32(sAl), bh = tc::smem_u32(sBh), bl = tc::smem_u32(sBl);

  const int64_t ntiles = (nsel + kTcRows - 1) / kTcRows;
  // row mode: v = this thread's block; coalesced mode: v = elements
  // tdep + ioff[i] of the tile (index i), base = the tile's first address
  float2 v[D2];
  int64_t tile = blockIdx.x;
  int64_t j = 0;
  bool live = false;
  float2* stage = reinterpret_cast<float2*>(sAl);   // coalesced mode: 128 x 2^m, row-swizzled
  float2* stage2 = reinterpret_cast<float2*>(sAh);  // coalesced mode: results
  auto sidx = [](int row, int l) { return row * D2 + (l ^ (row & (D2 - 1))); };
  auto gather = [&](int64_t t) {
    if constexpr (COAL) {
      j = deposit(t * kTcRows, fx);
#pragma unroll
      for (int i = 0; i < D2; ++i)
        v[i] = t * kTcRows + (trow | irow[i]) < nsel ? a[j + tdep + ioff[i]] : make_float2(0.f, 0.f);
    } else {
      const int64_t b = t * kTcRows + tid;
      live = b < nsel;
      j = live ? deposit(b, fx) : 0;
#pragma unroll
      for (int l = 0; l < D2; ++l) v[l] = live ? a[j + toff[l]] : make_float2(0.f, 0.f);
    }
  };
  if (tile < ntiles) gather(tile);
  uint32_t parity = 0;
  bool ok = true;
  for (; tile < ntiles; tile += gridDim.x) {
    if constexpr (COAL) {
      // elements to the staging buffer, then this thread's block back out
#pragma unroll
      for (int i = 0; i < D2; ++i) stage[sidx(trow | irow[i], tl | il[i])] = v[i];
      __syncthreads();
#pragma unroll
      for (int l = 0; l < D2; ++l) v[l] = stage[sidx(tid, l)];
    }
    // this thread's row of A = [Re v, Im v], split into TF32 hi and lo (in
    // coalesced mode lo only after every thread has read the staging area)
    float4 lo4[KD / 4];
#pragma unroll
    for (int kc = 0; kc < KD / 4; ++kc) {
      float x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = 4 * kc + i;
        x[i] = k < D2 ? v[k & (D2 - 1)].x : v[k & (D2 - 1)].y;
      }
      const float4 h = make_float4(tc::tf32_hi(x[0]), tc::tf32_hi(x[1]), tc::tf32_hi(x[2]), tc::tf32_hi(x[3]));
      lo4[kc] = make_float4(x[0] - h.x, x[1] - h.y, x[2] - h.z, x[3] - h.w);
      *reinterpret_cast<float4*>(&sAh[tc::at<kTcRows>(tid, 4 * kc)]) = h;
      if constexpr (!COAL) *reinterpret_cast<float4*>(&sAl[tc::at<kTcRows>(tid, 4 * kc)]) = lo4[kc];
    }
    if constexpr (COAL) {
      __syncthreads();
#pragma unroll
      for (int kc = 0; kc < KD / 4; ++kc) *reinterpret_cast<float4*>(&sAl[tc::at<kTcRows>(tid, 4 * kc)]) = lo4[kc];
    }
    const int64_t jcur = j;
    const bool lcur = live;
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      // lo*hi + hi*lo + hi*hi; K advances 8 (two core matrices) per MMA
      const uint32_t as[3] = {al, ah, ah}, bs[3] = {bh, bl, bh};
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int kk = 0; kk < KD / 8; ++kk)
          tc::mma_tf32(tmem, tc::desc(as[q] + kk * 2 * (kTcRows * 16), kTcRows * 16, 128),
                       tc::desc(bs[q] + kk * 2 * (ND * 16), ND * 16, 128), kIdesc, (q | kk) != 0);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a));
    }
    // next tile's amplitudes while the tensor cores work
    if (tile + gridDim.x < ntiles) gather(tile + gridDim.x);
    const bool done = tc::mbar_wait(bar_a, parity);
    parity ^= 1u;
    if (__syncthreads_or(!done)) {
      ok = false;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    uint32_t r[ND];
    const uint32_t tmem_row = tmem + (uint32_t(warp * 32) << 16);
    tc::ld32<0>(tmem_row, r);
    if constexpr (ND > 32) tc::ld32<32>(tmem_row + 32u, r);
    tc::wait_ld(r);
    if constexpr (COAL) {
      // this thread's block to the results area, then elements out in
      // address order
#pragma unroll
      for (int n = 0; n < D2; ++n) stage2[sidx(tid, n)] = make_float2(__uint_as_float(r[n]), __uint_as_float(r[D2 + n]));
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
#pragma unroll
      for (int i = 0; i < D2; ++i) {
        const int row = trow | irow[i];
        if (tile * kTcRows + row < nsel) a[jcur + tdep + ioff[i]] = stage2[sidx(row, tl | il[i])];
      }
    } else {
      if (lcur) {
#pragma unroll
        for (int n = 0; n < D2; ++n)
          a[jcur + toff[n]] = make_float2(__uint_as_float(r[n]), __uint_as_float(r[D2 + n]));
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, 1u);
    tc::mbar_wait(bar_a, parity ^ 1u);  // the outstanding commit, bounded
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(ND)));
}

// ------------------------------------------------------------ staged form
// The staged kernel (registers with at least 7 free qubits, nsel >= 128):
// a tile is the 128 x 2^m amplitudes whose enumeration bits (the 7 lowest
// free qubits and the targets, ascending: pos[], role[]) vary, i.e. the
// address pattern tile base + dep(e), e < 2^(7+m).  Tiles are copied in
// address order (16-byte cp.async chunks, coalesced whatever the targets)
// into one of two shared-memory stages, two tiles ahead of the one being
// worked.  G threads share a block (row): each reads its 2^m / G elements
// out of the stage, splits them into TF32 hi and lo and writes them to the
// row's tensor-memory lane as its columns of the A operand (tcgen05.st);
// the MMAs read A from tensor memory and B from shared memory, and each
// thread stores its 2^m / G outputs straight from registers.  Shared
// memory: the two stages and B hi / lo; tensor memory: the accumulator
// (2^(m+1) columns) and A hi / lo (2^(m+1) each).  With 2^m / G = 16
// elements a thread, m = 5 runs 256 threads (two CTAs, 16 warps an SM; the
// tensor memory holds two) and m = 4 runs 128 (four CTAs an SM).
template <int MT>
__host__ __device__ constexpr int tcs_group() {
  return MT == 5 ? 2 : 1;
}

template <int MT>
__host__ __device__ constexpr uint32_t tcs_tmem_cols() {
  return (6u << MT) <= 32u ? 32u : (6u << MT) <= 64u ? 64u : (6u << MT) <= 128u ? 128u : (6u << MT) <= 256u ? 256u : 512u;
}

template <int MT>
__host__ __device__ constexpr size_t tcs_stage_bytes() {
  return size_t(kTcRows) * (1 << MT) * 8;
}

// Copy chunks (16 bytes) per thread per tile.
template <int MT>
__host__ __device__ constexpr int tcs_rounds() {
  return (1 << MT) / (2 * tcs_group<MT>());
}

// Shared memory of the staged kernel: two stages, B hi / lo, the target
// offsets (int64 per combination), the address offsets and chunk positions
// of the copy rounds (int64, uint16), the mbarrier and the tensor-memory
// slot.
template <int MT>
__host__ __device__ constexpr size_t tcs_smem_bytes() {
  return 2 * tcs_stage_bytes<MT>() + size_t(2) * (2 << MT) * (2 << MT) * 4 + 8 * (1 << MT) + 10 * tcs_rounds<MT>() + 64;
}

// MODE 0: the lowest five row bits are qubits 0..4 (targets and controls
// above them), so a warp's 32 rows are 32 consecutive amplitudes: results
// are stored straight from registers, coalesced, and the stage is refilled
// as soon as A is in tensor memory.  MODE 1 and 2: a warp's rows are far
// apart, so direct stores would touch up to 32 lines an instruction: the
// results go back into the tile's stage (to the positions their inputs
// came from) and leave it in address order, 16-byte chunks, the mirror of
// the copy in; the stage is refilled after that.  MODE 2: enumeration bit
// 0 is target 0 at qubit 0 (targets sorted ascending), so elements 2l,
// 2l + 1 of a row are adjacent: read and written as one 16-byte access.
template <int MT, int MODE>
__global__ void __launch_bounds__(kTcRows * tcs_group<MT>())
    k_sv_multi_tcs(float2* __restrict__ a, int64_t nsel, const __grid_constant__ Fixed fx,
                   const __grid_constant__ TcParams<MT> p, unsigned* status) {
  constexpr bool PAIR = MODE == 2, DIRECT = MODE == 0;
  constexpr int D2 = 1 << MT, KD = 2 * D2, ND = 2 * D2, E = 7 + MT;
  constexpr int G = tcs_group<MT>(), T = kTcRows * G, LT = G == 2 ? 8 : 7;  // T = 2^LT threads
  constexpr int LH = D2 / G;       // elements (and outputs) of a row per thread
  constexpr int NR = tcs_rounds<MT>();
  static_assert(MT >= 4 && MT <= 5 && LH == 16, "16 columns a thread per tensor-memory access");
  static_assert(NR == 1 << (E - 1 - LT), "copy rounds");
  constexpr uint32_t kStage = uint32_t(tcs_stage_bytes<MT>()), kB = ND * KD * 4;
  constexpr uint32_t kCols = tcs_tmem_cols<MT>();
  constexpr uint32_t kIdesc = tc::idesc_tf32(kTcRows, ND);
  static_assert(ND + 2 * KD <= int(kCols), "tensor-memory layout");
  extern __shared__ __align__(1024) uint8_t smem[];
  float* sBh = reinterpret_cast<float*>(smem + 2 * kStage);
  float* sBl = reinterpret_cast<float*>(smem + 2 * kStage + kB);
  int64_t* ldep = reinterpret_cast<int64_t*>(smem + 2 * kStage + 2 * kB);  // [D2] address offset of combination l
  int64_t* cdep = ldep + D2;                                               // [NR] address offset of round i
  uint16_t* cpos = reinterpret_cast<uint16_t*>(cdep + NR);                 // [NR] chunk position of round i
  constexpr uint32_t kBar = (2 * kStage + 2 * kB + 8 * D2 + 10 * NR + 7) / 8 * 8;
  static_assert(kBar + 16 <= tcs_smem_bytes<MT>(), "shared-memory layout");
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, row = tid & (kTcRows - 1), hf = tid / kTcRows;

  // enumeration index of row bit b and of target u
  int krow[7], ktg[MT];
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int r = p.role[k];
#pragma unroll
    for (int u = 0; u < MT; ++u)
      if (r == (0x80 | u)) ktg[u] = k;
#pragma unroll
    for (int b = 0; b < 7; ++b)
      if (r == b) krow[b] = k;
  }
  // this thread's row: element bits (erow), their stage position and their
  // address offset; its elements hf * LH + i: stage positions lp[i]
  uint32_t erow = 0;
  int64_t rdep = 0;
#pragma unroll
  for (int b = 0; b < 7; ++b)
    if ((row >> b) & 1) {
      erow |= 1u << krow[b];
      rdep += int64_t(1) << p.pos[krow[b]];
    }
  const uint32_t prow = tc::elem_pos(erow);
  uint32_t lp[LH];
#pragma unroll
  for (int i = 0; i < LH; ++i) {
    const int l = hf * LH + i;
    uint32_t el = 0;
#pragma unroll
    for (int u = 0; u < MT; ++u)
      if ((l >> u) & 1) el |= 1u << ktg[u];
    lp[i] = prow ^ tc::elem_pos(el);
  }
  // copy chunks tid + T i: element bits 1..LT from tid (address ctdep,
  // position chunk_swz(tid)), bits LT + 1.. from i (cdep[i], cpos[i])
  int64_t ctdep = 0;
#pragma unroll
  for (int k = 1; k <= LT; ++k)
    if ((tid >> (k - 1)) & 1) ctdep += int64_t(1) << p.pos[k];
  const uint32_t ctpos = tc::chunk_swz(uint32_t(tid));
  const int64_t half = int64_t(1) << p.pos[0];  // address step of element bit 0 (split copies)

  // B = [[Re U^T, Im U^T], [-Im U^T, Re U^T]] stored N x K (row n = output
  // column): row n < D2 gives Re w[n], row D2 + n gives Im w[n].
  for (int e = tid; e < ND * KD; e += T) {
    const int n = e / KD, k = e % KD;
    const float2 u = p.u[(n & (D2 - 1)) * D2 + (k & (D2 - 1))];
    const float v = n < D2 ? (k < D2 ? u.x : -u.y) : (k < D2 ? u.y : u.x);
    const float h = tc::tf32_hi(v);
    sBh[tc::at<ND>(n, k)] = h;
    sBl[tc::at<ND>(n, k)] = v - h;
  }
  if (tid < D2) {
    int64_t d = 0;
#pragma unroll
    for (int u = 0; u < MT; ++u)
      if ((tid >> u) & 1) d += int64_t(1) << p.pos[ktg[u]];
    ldep[tid] = d;
  }
  if (tid < NR) {
    int64_t d = 0;
    for (int k = LT + 1; k < E; ++k)
      if ((tid >> (k - LT - 1)) & 1) d += int64_t(1) << p.pos[k];
    cdep[tid] = d;
    cpos[tid] = uint16_t(tc::chunk_swz(uint32_t(tid) << LT));
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tslot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");  // B, written by the threads, read by the MMAs
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t bar_a = tc::smem_u32(bar);
  const uint32_t bh = tc::smem_u32(sBh), bl = tc::smem_u32(sBl);
  const uint32_t stage0 = tc::smem_u32(smem);
  const uint32_t trow = tmem + (uint32_t((warp & 3) * 32) << 16);  // this warp's lanes (its rows)
  const uint32_t cre = uint32_t(hf * LH), cim = uint32_t(D2 + hf * LH);  // this thread's columns
  const bool split = p.split != 0;

  const int64_t ntiles = nsel / kTcRows;  // nsel is a power of two >= 128
  // copies of tile t into stage s (every thread its NR chunks)
  auto issue = [&](int64_t t, int s) {
    const float2* src = a + deposit(t * kTcRows, fx) + ctdep;
    const uint32_t dst = stage0 + uint32_t(s) * kStage;
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const uint32_t d = dst + ((ctpos ^ cpos[i]) << 4);
      const float2* sp = src + cdep[i];
      if (!split) {
        tc::cp16(d, sp);
      } else {
        tc::cp8(d, sp);
        tc::cp8(d + 8, sp + half);
      }
    }
  };
  int64_t tile = blockIdx.x;
  const int64_t step = gridDim.x;
  if (tile < ntiles) issue(tile, 0);
  tc::cp_commit();
  if (tile + step < ntiles) issue(tile + step, 1);
  tc::cp_commit();
  uint32_t parity = 0;
  bool ok = true;
  int s = 0;
  for (; tile < ntiles; tile += step, s ^= 1) {
    tc::cp_wait<1>();  // this thread's copies of this tile
    __syncthreads();   // everyone's
    const float2* st = reinterpret_cast<const float2*>(smem + uint32_t(s) * kStage);
    float2 v[LH];
    if constexpr (PAIR) {
#pragma unroll
      for (int i = 0; i < LH; i += 2) {
        const float4 q = *reinterpret_cast<const float4*>(st + lp[i]);
        v[i] = make_float2(q.x, q.y);
        v[i + 1] = make_float2(q.z, q.w);
      }
    } else {
#pragma unroll
      for (int i = 0; i < LH; ++i) v[i] = st[lp[i]];
    }
    // this thread's columns of A = [Re v, Im v] as TF32 hi and lo: hi at
    // ND.., lo at ND + KD..
    {
      uint32_t h[16], lo[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float hx = tc::tf32_hi(v[i].x);
        h[i] = __float_as_uint(hx);
        lo[i] = __float_as_uint(v[i].x - hx);
      }
      tc::st16(trow + uint32_t(ND) + cre, h);
      tc::st16(trow + uint32_t(ND + KD) + cre, lo);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float hy = tc::tf32_hi(v[i].y);
        h[i] = __float_as_uint(hy);
        lo[i] = __float_as_uint(v[i].y - hy);
      }
      tc::st16(trow + uint32_t(ND) + cim, h);
      tc::st16(trow + uint32_t(ND + KD) + cim, lo);
    }
    tc::wait_st();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // A complete; the stage is free; last tile's accumulator reads done
    asm volatile("tcgen05.fence::after_thread_sync;");
    if constexpr (DIRECT) {
      if (tile + 2 * step < ntiles) issue(tile + 2 * step, s);
      tc::cp_commit();
    }
    if (tid == 0) {
      // lo*hi + hi*lo + hi*hi; K advances 8 columns (two core matrices of B)
      const uint32_t as[3] = {uint32_t(ND + KD), uint32_t(ND), uint32_t(ND)}, bs[3] = {bh, bl, bh};
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int kk = 0; kk < KD / 8; ++kk)
          tc::mma_tf32_ts(tmem, tmem + as[q] + uint32_t(kk * 8), tc::desc(bs[q] + kk * 2 * (ND * 16), ND * 16, 128),
                          kIdesc, (q | kk) != 0);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a));
    }
    const int64_t j = deposit(tile * kTcRows, fx) + rdep;
    const bool done = tc::mbar_wait(bar_a, parity);
    parity ^= 1u;
    if (__syncthreads_or(!done)) {
      ok = false;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    uint32_t r[32];
    tc::ld16<0>(trow + cre, r);
    tc::ld16<16>(trow + cim, r);
    tc::wait_ld(r);
    if constexpr (DIRECT) {
      float2* dst = a + j;
#pragma unroll
      for (int i = 0; i < LH; ++i)
        dst[ldep[hf * LH + i]] = make_float2(__uint_as_float(r[i]), __uint_as_float(r[16 + i]));
    } else {
      float2* so = reinterpret_cast<float2*>(smem + uint32_t(s) * kStage);
      if constexpr (PAIR) {
#pragma unroll
        for (int i = 0; i < LH; i += 2)
          *reinterpret_cast<float4*>(so + lp[i]) = make_float4(__uint_as_float(r[i]), __uint_as_float(r[16 + i]),
                                                               __uint_as_float(r[i + 1]), __uint_as_float(r[16 + i + 1]));
      } else {
#pragma unroll
        for (int i = 0; i < LH; ++i) so[lp[i]] = make_float2(__uint_as_float(r[i]), __uint_as_float(r[16 + i]));
      }
      __syncthreads();
      float2* dst = a + (j - rdep) + ctdep;  // the tile's base + this thread's chunk bits
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        const float4 q = *reinterpret_cast<const float4*>(so + 2 * (ctpos ^ cpos[i]));
        float2* dp = dst + cdep[i];
        if (!split) {
          *reinterpret_cast<float4*>(dp) = q;
        } else {
          dp[0] = make_float2(q.x, q.y);
          dp[half] = make_float2(q.z, q.w);
        }
      }
      __syncthreads();  // the stage is read out: refill it
      if (tile + 2 * step < ntiles) issue(tile + 2 * step, s);
      tc::cp_commit();
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  tc::cp_wait<0>();  // no copy still in flight when the CTA ends
  if (!ok) {
    if (tid == 0) atomicOr(status, 1u);
    tc::mbar_wait(bar_a, parity ^ 1u);  // the outstanding commit, bounded
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// Diagnostic: the bounded wait of k_sv_multi_tc on an mbarrier that nothing
// arrives on, so it runs out after max_ns and reports through the status
// word exactly as the tensor-core pass would.
__global__ void k_wait_probe(unsigned* status, uint64_t max_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  const bool done = tc::mbar_wait(tc::smem_u32(&bar), 0, max_ns);
  if (__syncthreads_or(!done) && threadIdx.x == 0) atomicOr(status, 1u);
}

}  // namespace qs
