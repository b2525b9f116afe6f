// Fused tile kernel: one HBM round trip applies a whole pass of operations.
//
// A pass fixes k "tile qubits" Q (always the L lowest qubits, for
// contiguous 2^L-amplitude chunks, plus k-L others).  For every assignment
// of the remaining bits (one tile) the 2^k amplitudes are loaded into shared
// memory, every operation of the pass is applied, and the tile is written
// back.  Non-diagonal operations must act on tile qubits; diagonal ones and
// controls may sit anywhere (outside the tile they are a per-tile
// predicate).
//
// Inside a tile the pass is split into stages.  A stage names R "register
// bits" of the local index; each thread holds the 2^R amplitudes that
// differ only in those bits, applies the stage's operations in registers,
// and writes them back to shared memory.  Pair updates (Eq. 1) on a
// register bit, and quad updates on two register bits, need no further
// shared-memory traffic.  The pass's operation list is copied into shared
// memory once per CTA, so decoding an operation costs shared-memory
// broadcasts only.
#pragma once
#include "fused_arith.cuh"
#include "pass_kernels.cuh"

namespace qs {


// Mask of register indices j with bit i clear, as a bit set over j (R <= 5).
__constant__ uint32_t c_bit_clear[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu,
                                        0x0000FFFFu};

// True when the set `f` of register indices is NOT invariant under toggling
// index bit i, i.e. a diagonal op with support f does not commute with a
// pair update on register bit i.
__device__ __forceinline__ bool depends_on_bit(uint32_t f, int i) {
  const uint32_t m = c_bit_clear[i];
  const int s = 1 << i;
  return ((((f >> s) & m) | ((f & m) << s)) != f);
}

__device__ __forceinline__ int bit_value(uint8_t src, uint8_t pos, int j, uint32_t tlocal,
                                         uint64_t tglobal) {
  if (src == BS_REG) return (j >> pos) & 1;
  if (src == BS_LOCAL) return int((tlocal >> pos) & 1u);
  return int((tglobal >> pos) & 1u);
}

// Applies one operation (dispatch code `code`, register controls `rmask`)
// to the thread's 2^R register amplitudes; sign flips only update the
// pending mask `flips`.  tlocal: this thread's local index with the register
// bits zero; tglobal: the tile's global base (tile bits zero).
template <class A, int R>
__device__ __forceinline__ void run_op(typename A::Cplx (&v)[1 << R], const FOp& op, uint32_t code,
                                       uint32_t rmask, uint32_t tlocal, uint64_t tglobal,
                                       uint32_t& flips) {
#define QS_BIT_CASE(FAM, S, ...) \
  case FAM * kCodeSlots + S: if constexpr (R > S) { constexpr int I = S; __VA_ARGS__; } break;
#define QS_BIT_CASES(FAM, ...)                                                              \
  QS_BIT_CASE(FAM, 0, __VA_ARGS__) QS_BIT_CASE(FAM, 1, __VA_ARGS__) QS_BIT_CASE(FAM, 2, __VA_ARGS__) \
  QS_BIT_CASE(FAM, 3, __VA_ARGS__) QS_BIT_CASE(FAM, 4, __VA_ARGS__)
#define QS_PAIR_CASE(FAM, S, A_, B_, ...)                                   \
  case FAM * kCodeSlots + S:                                                 \
    if constexpr (R > B_) { constexpr int IA = A_, IB = B_; __VA_ARGS__; } \
    break;
#define QS_PAIR_CASES(FAM, ...)                                                                   \
  QS_PAIR_CASE(FAM, 0, 0, 1, __VA_ARGS__) QS_PAIR_CASE(FAM, 1, 0, 2, __VA_ARGS__)                 \
  QS_PAIR_CASE(FAM, 2, 0, 3, __VA_ARGS__) QS_PAIR_CASE(FAM, 3, 0, 4, __VA_ARGS__)                 \
  QS_PAIR_CASE(FAM, 4, 1, 2, __VA_ARGS__) QS_PAIR_CASE(FAM, 5, 1, 3, __VA_ARGS__)                 \
  QS_PAIR_CASE(FAM, 6, 1, 4, __VA_ARGS__) QS_PAIR_CASE(FAM, 7, 2, 3, __VA_ARGS__)                 \
  QS_PAIR_CASE(FAM, 8, 2, 4, __VA_ARGS__) QS_PAIR_CASE(FAM, 9, 3, 4, __VA_ARGS__)
#define QS_SIDE_CASE(FAM, I_, J_, K_, C_)                                      \
  case FAM * kCodeSlots + I_ * 4 + J_:                                          \
    if constexpr (A::kSide && R == 4) pair_side_on_bit<A, R, K_, C_, I_, J_>(v, op); \
    break;
#define QS_SIDE_CASES(FAM, K_, C_)                                                                    \
  QS_SIDE_CASE(FAM, 0, 1, K_, C_) QS_SIDE_CASE(FAM, 0, 2, K_, C_) QS_SIDE_CASE(FAM, 0, 3, K_, C_)     \
  QS_SIDE_CASE(FAM, 1, 0, K_, C_) QS_SIDE_CASE(FAM, 1, 2, K_, C_) QS_SIDE_CASE(FAM, 1, 3, K_, C_)     \
  QS_SIDE_CASE(FAM, 2, 0, K_, C_) QS_SIDE_CASE(FAM, 2, 1, K_, C_) QS_SIDE_CASE(FAM, 2, 3, K_, C_)     \
  QS_SIDE_CASE(FAM, 3, 0, K_, C_) QS_SIDE_CASE(FAM, 3, 1, K_, C_) QS_SIDE_CASE(FAM, 3, 2, K_, C_)
  switch (code) {
    QS_SIDE_CASES(FC_H_SIDE, PK_H, false)
    QS_SIDE_CASES(FC_SX_SIDE, PK_SX, false)
    QS_SIDE_CASES(FC_SX_C_SIDE, PK_SX, true)
    QS_SIDE_CASES(FC_SY_SIDE, PK_SY, false)
#undef QS_SIDE_CASES
#undef QS_SIDE_CASE
    QS_BIT_CASES(FC_GEN, (pair_on_bit<A, R, PK_GEN, false, true, I>(v, rmask, op)))
    QS_BIT_CASES(FC_GEN_C, (pair_on_bit<A, R, PK_GEN, true, true, I>(v, rmask, op)))
    QS_BIT_CASES(FC_H, (pair_on_bit<A, R, PK_H, false, false, I>(v, rmask, op)))
    QS_BIT_CASES(FC_SX, (pair_on_bit<A, R, PK_SX, false, false, I>(v, rmask, op)))
    QS_BIT_CASES(FC_SX_C, (pair_on_bit<A, R, PK_SX, true, false, I>(v, rmask, op)))
    QS_BIT_CASES(FC_SY, (pair_on_bit<A, R, PK_SY, false, false, I>(v, rmask, op)))
    QS_BIT_CASES(FC_X, (pair_on_bit<A, R, PK_X, false, true, I>(v, rmask, op)))
    QS_BIT_CASES(FC_PHASE_BIT, (phase_on_bit<A, R, I>(v, op)))
    QS_PAIR_CASES(FC_DEPOL, (depol_on_bits<A, R, IA, IB>(v, op)))
    QS_PAIR_CASES(FC_DEPH_PAIR, (deph_on_bits<A, R, IA, IB>(v, op)))
    QS_PAIR_CASES(FC_OFFPH, (offph_on_bits<A, R, IA, IB>(v, op)))
    QS_BIT_CASES(FC_MULI_BIT, (muli_on_bit<A, R, I>(v)))
    QS_BIT_CASES(FC_SHEAR, (shear_on_bit<A, R, I, 0>(v, op)))
    QS_BIT_CASES(FC_SHEAR2, (shear_on_bit<A, R, I, 1>(v, op)))
    QS_BIT_CASES(FC_PHASEU_BIT, (phaseu_on_bit<A, R, I>(v, op)))
    case FC_PHASEU_ALL * kCodeSlots:
#pragma unroll
      for (int j = 0; j < (1 << R); ++j) v[j] = A::phase_u(v[j], op);
      break;
    case FC_MULI_ALL * kCodeSlots:
#pragma unroll
      for (int j = 0; j < (1 << R); ++j) v[j] = A::mul_i(v[j]);
      break;
    case FC_MULI_MASK * kCodeSlots: {
      const uint32_t touch = op.c.u[15];
#pragma unroll
      for (int j = 0; j < (1 << R); ++j)
        if ((touch >> j) & 1u) v[j] = A::mul_i(v[j]);
      break;
    }
#undef QS_PAIR_CASES
#undef QS_PAIR_CASE
#undef QS_BIT_CASES
#undef QS_BIT_CASE
    case FC_PHASE_ALL * kCodeSlots:
#pragma unroll
      for (int j = 0; j < (1 << R); ++j) v[j] = A::phase(v[j], op);
      break;
    case FC_PHASE_MASK * kCodeSlots: {
      const uint32_t touch = op.c.u[15];
#pragma unroll
      for (int j = 0; j < (1 << R); ++j)
        if ((touch >> j) & 1u) v[j] = A::phase(v[j], op);
      break;
    }
    case FC_SIGN * kCodeSlots: flips ^= op.c.u[15]; break;
    case FC_DEPH * kCodeSlots:
#pragma unroll
      for (int j = 0; j < (1 << R); ++j)
        if (bit_value(op.asrc, op.apos, j, tlocal, tglobal) !=
            bit_value(op.bsrc, op.bpos, j, tlocal, tglobal))
          v[j] = A::scale(v[j], op, 0);
      break;
    case FC_SCALE * kCodeSlots:
#pragma unroll
      for (int j = 0; j < (1 << R); ++j) v[j] = A::phase(v[j], op);
      break;
    default: break;
  }
}

// A tile held in the CTA's own shared memory: element l at t[l].
template <class A>
struct LocalTile {
  typename A::Cplx* t;
  __device__ __forceinline__ typename A::Cplx load(uint32_t l) const { return t[l]; }
  __device__ __forceinline__ void store(uint32_t l, const typename A::Cplx& v) const { t[l] = v; }
};

// One stage of a pass for one thread: its 2^R register amplitudes from the
// tile, the stage's operations, and back.  tidx: the thread's index among
// the tile's 2^(k-R) stage threads; base: the tile's global base (tile bits
// zero); ops: the pass's op list.
template <class A, int R, class Tile>
__device__ __forceinline__ void run_stage(const Tile& tile, const FStage& st, const FOp* ops, uint32_t tidx,
                                          uint64_t base) {
  using Cplx = typename A::Cplx;
  uint32_t poff[R];
  uint32_t pm = 0, cpm = 0;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    poff[i] = 1u << st.pbits[i];
    pm |= poff[i];
    // register bits in st.copy start as copies of their bit-0 half
    if ((st.copy >> i) & 1u) cpm |= poff[i];
  }
  // tlocal: tidx with a zero bit inserted at each register-bit
  // position (positions ascending), i.e. its bits spread over the local
  // positions not in pm
  uint32_t tlocal = tidx;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const uint32_t p = st.pbits[i];
    tlocal = ((tlocal >> p) << (p + 1)) | (tlocal & ((1u << p) - 1u));
  }
  Cplx v[1 << R];
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) {
    uint32_t off = 0;
#pragma unroll
    for (int i = 0; i < R; ++i)
      if (j & (1 << i)) off |= poff[i];
    v[j] = tile.load(tlocal | (off & ~cpm));
  }
  // Sign flips (CZ, multi-controlled phase flips) commute with every
  // diagonal op, and with a pair update on register bit i whenever the
  // flipped set is symmetric under toggling bit i; so they are collected
  // as a per-thread mask over the register amplitudes and applied only
  // before an op they do not commute with, or at the end of the stage.
  uint32_t flips = 0;
  // code, flags and rmask share one word (read one op ahead); kind,
  // conj, i0, i1 another
  const int oe = st.op_end;
  uint32_t wnext = st.op_begin < oe ? *reinterpret_cast<const uint32_t*>(&ops[st.op_begin].code) : 0u;
  for (int o = st.op_begin; o < oe; ++o) {
    const FOp& op = ops[o];
    const uint32_t w = wnext;
    wnext = o + 1 < oe ? *reinterpret_cast<const uint32_t*>(&ops[o + 1].code) : 0u;
    const uint32_t flags = (w >> 16) & 0xFFu;
    if ((flags & FF_COND) &&
        ((tlocal & op.lmask) != op.lmask || (base & op.gmask) != op.gmask))
      continue;
    if ((flags & FF_FLIP) && flips) {
      const uint32_t w0 = *reinterpret_cast<const uint32_t*>(&op);
      if (depends_on_bit(flips, (w0 >> 16) & 0xFFu) ||
          ((flags & FF_TWO) && depends_on_bit(flips, w0 >> 24))) {
#pragma unroll
        for (int j = 0; j < (1 << R); ++j)
          if ((flips >> j) & 1u) v[j] = A::negate(v[j]);
        flips = 0;
      }
    }
    if ((w & 0xFFFFu) == FC_SIGN * kCodeSlots) {
      flips ^= op.c.u[15];
      continue;
    }
    run_op<A, R>(v, op, w & 0xFFFFu, op.rmask, tlocal, base, flips);
  }
  if (flips) {
#pragma unroll
    for (int j = 0; j < (1 << R); ++j)
      if ((flips >> j) & 1u) v[j] = A::negate(v[j]);
  }
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) {
    uint32_t off = 0;
#pragma unroll
    for (int i = 0; i < R; ++i)
      if (j & (1 << i)) off |= poff[i];
    tile.store(tlocal | off, v[j]);
  }
}

// Shared-memory bytes of a pass launch.
template <class A>
__host__ __device__ inline size_t fused_smem_bytes(int k, int L, int nops, int nstages) {
  return sizeof(typename A::Cplx) * (size_t(1) << k) + sizeof(int64_t) * (size_t(1) << (k - L)) +
         sizeof(FOp) * size_t(nops) + sizeof(FStage) * size_t(nstages);
}

// ------------------------------------------------------------------ kernel
constexpr int kFusedThreads = 256;
// Resident CTAs per SM of the fused kernels: 2 (128 registers a thread) for
// R >= 4; 3 (85 registers) for R = 3, whose 8 register amplitudes leave room
// (measured for FP64: no faster than R = 4, which is the configuration used).
__host__ __device__ constexpr int fused_ctas_per_sm(int R) { return R <= 3 ? 3 : 2; }
// Global accesses per thread in one round of a tile load or store.  The
// single-register kernel runs 2^(k-R) threads on a 2^k tile, so each thread
// owns exactly 2^R amplitudes: 2^R complex128 accesses or 2^(R-1) float4
// accesses of two complex64.  It issues all of them at once (one round, no
// bounds test needed: the round covers the tile exactly; the register
// amplitudes are not live yet).  The batched kernel runs 256 threads on
// tiles of any size with bounds tests, 8 accesses a round.
template <class A, int R, bool GENERAL>
__host__ __device__ constexpr int tile_access_depth() {
  return GENERAL ? 8 : (sizeof(typename A::Store) == 8 ? (1 << (R - 1)) : (1 << R));
}

// Shared-memory layout of a pass: tile, chunk offsets, op list, stage list.
template <class A>
struct PassSmem {
  typename A::Cplx* tile;
  int64_t* choff;
  FOp* ops;
  FStage* st;
};

template <class A>
__device__ __forceinline__ PassSmem<A> pass_smem(unsigned char* raw, int kmax, int Lmin, int opmax) {
  PassSmem<A> m;
  m.tile = reinterpret_cast<typename A::Cplx*>(raw);
  m.choff = reinterpret_cast<int64_t*>(raw + sizeof(typename A::Cplx) * (size_t(1) << kmax));
  m.ops = reinterpret_cast<FOp*>(m.choff + (1 << (kmax - Lmin)));
  m.st = reinterpret_cast<FStage*>(m.ops + opmax);
  return m;
}

// Copies a pass's chunk-offset table, op list and stage list into shared
// memory (all threads; caller synchronises).
template <class A>
__device__ __forceinline__ void load_pass(const FPass& P, const FOp* __restrict__ ops,
                                          const FStage* __restrict__ stages, PassSmem<A>& m) {
  const int nchunk = 1 << (P.k - P.L);
  for (int c = threadIdx.x; c < nchunk; c += blockDim.x) {
    int64_t off = 0;
    for (int i = 0; i < P.k - P.L; ++i)
      if ((c >> i) & 1) off |= int64_t(1) << P.q[P.L + i];
    m.choff[c] = off;
  }
  const uint64_t* src = reinterpret_cast<const uint64_t*>(ops + P.op_begin);
  uint64_t* dst = reinterpret_cast<uint64_t*>(m.ops);
  const int nw = P.op_count * int(sizeof(FOp) / 8);
  for (int w = threadIdx.x; w < nw; w += blockDim.x) dst[w] = src[w];
  const uint64_t* ss = reinterpret_cast<const uint64_t*>(stages + P.stage_begin);
  uint64_t* sd = reinterpret_cast<uint64_t*>(m.st);
  const int ns = (P.stage_end - P.stage_begin) * int(sizeof(FStage) / 8);
  for (int w = threadIdx.x; w < ns; w += blockDim.x) sd[w] = ss[w];
}

// Applies pass P to tile tau of the register g: load (or generate |0...0>),
// run the stages, store.  2^(k-R) threads work on the stages; all threads of
// the block take part in loads, stores and barriers.  GENERAL = false is the
// single-register launch, where blockDim = 2^(k-R) and no pass generates
// |0...0>, so those checks compile away.
// CG: tile loads bypass L1 (ld.global.cg), for a kernel that reads
// amplitudes other CTAs wrote earlier in the same launch (L1 is not coherent
// across SMs, and this SM may hold older copies of the same lines).
template <class A, int R, bool GENERAL, bool CG = false>
__device__ __forceinline__ void process_tile(typename A::Store* __restrict__ g, const FPass& P,
                                             int64_t tau, PassSmem<A>& m) {
  using Cplx = typename A::Cplx;
  using Store = typename A::Store;
  const int k = P.k, L = P.L;
  const int ntile = 1 << k;
  const int lmask_low = (1 << L) - 1;
  const int nst = P.stage_end - P.stage_begin;
  const int active = 1 << (k - R);
  constexpr int kDepth = tile_access_depth<A, R, GENERAL>();
  // global base of the tile: the bits of tau in the non-tile positions
  int64_t base = tau;
  for (int i = 0; i < k; ++i) {
    const int p = P.q[i];
    base = ((base >> p) << (p + 1)) | (base & ((int64_t(1) << p) - 1));
  }
  if (GENERAL && P.init) {
    for (int l = threadIdx.x; l < ntile; l += blockDim.x) {
      Store z;
      z.x = 0;
      z.y = 0;
      if (base == 0 && l == 0) z.x = 1;
      m.tile[l] = A::from_store(z);
    }
  } else if constexpr (sizeof(Store) == 8) {
    // complex64: two amplitudes per 16-byte access (chunks of 2^L >= 2
    // contiguous amplitudes start at even indices)
    const int npair = ntile >> 1;
    const float4* g4 = reinterpret_cast<const float4*>(g);
    float4* t4 = reinterpret_cast<float4*>(m.tile);
    for (int e0 = threadIdx.x; e0 < npair; e0 += blockDim.x * kDepth) {
      float4 t[kDepth];
#pragma unroll
      for (int u = 0; u < kDepth; ++u) {
        const int l = 2 * (e0 + u * blockDim.x);
        if (!GENERAL || l < ntile) {
          const float4* src = g4 + ((base + m.choff[l >> L] + (l & lmask_low)) >> 1);
          if constexpr (CG) t[u] = __ldcg(src);
          else t[u] = *src;
        }
      }
#pragma unroll
      for (int u = 0; u < kDepth; ++u) {
        const int e = e0 + u * blockDim.x;
        if (!GENERAL || e < npair) t4[e] = t[u];
      }
    }
  } else {
    // load: kDepth independent loads in flight per thread
    for (int l0 = threadIdx.x; l0 < ntile; l0 += blockDim.x * kDepth) {
      Store t[kDepth];
#pragma unroll
      for (int u = 0; u < kDepth; ++u) {
        const int l = l0 + u * blockDim.x;
        if (!GENERAL || l < ntile) {
          const Store* src = g + (base + m.choff[l >> L] + (l & lmask_low));
          if constexpr (CG) t[u] = __ldcg(src);
          else t[u] = *src;
        }
      }
#pragma unroll
      for (int u = 0; u < kDepth; ++u) {
        const int l = l0 + u * blockDim.x;
        if (!GENERAL || l < ntile) m.tile[l] = A::from_store(t[u]);
      }
    }
  }
  __syncthreads();
  for (int s = 0; s < nst; ++s) {
    if (!GENERAL || int(threadIdx.x) < active)
      run_stage<A, R>(LocalTile<A>{m.tile}, m.st[s], m.ops, threadIdx.x, uint64_t(base));
    __syncthreads();
  }
  // store
  if constexpr (sizeof(Store) == 8) {
    const int npair = ntile >> 1;
    float4* g4 = reinterpret_cast<float4*>(g);
    const float4* t4 = reinterpret_cast<const float4*>(m.tile);
    for (int e0 = threadIdx.x; e0 < npair; e0 += blockDim.x * kDepth) {
#pragma unroll
      for (int u = 0; u < kDepth; ++u) {
        const int e = e0 + u * blockDim.x;
        if (!GENERAL || e < npair) g4[(base + m.choff[(2 * e) >> L] + ((2 * e) & lmask_low)) >> 1] = t4[e];
      }
    }
  } else {
    for (int l0 = threadIdx.x; l0 < ntile; l0 += blockDim.x * kDepth) {
#pragma unroll
      for (int u = 0; u < kDepth; ++u) {
        const int l = l0 + u * blockDim.x;
        if (!GENERAL || l < ntile) g[base + m.choff[l >> L] + (l & lmask_low)] = A::to_store(m.tile[l]);
      }
    }
  }
  __syncthreads();
}

// One pass over every tile of one register.
template <class A, int R>
__global__ void __launch_bounds__(kFusedThreads, fused_ctas_per_sm(R))
    k_fused(typename A::Store* __restrict__ g, const __grid_constant__ FPass P,
            const FOp* __restrict__ ops, const FStage* __restrict__ stages) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PassSmem<A> m = pass_smem<A>(smem_raw, P.k, P.L, P.op_count);
  load_pass<A>(P, ops, stages, m);
  __syncthreads();
  for (int64_t tau = blockIdx.x; tau < P.ntiles; tau += gridDim.x) process_tile<A, R, false>(g, P, tau, m);
}

// ------------------------------------------------------------ cluster form
// A pass over a register that is a single tile (2^k amplitudes) runs on one
// CTA in the kernel above, i.e. on one SM.  Here it runs on a cluster of C
// CTAs (C SMs): CTA r of the cluster holds tile elements r 2^(k-c) ..
// (r + 1) 2^(k-c) - 1 (c = log2 C) in its shared memory and runs stage
// threads r T .. (r + 1) T - 1 (T = 2^(k-R-c)).  A stage whose register
// bits all lie below bit k - c keeps every thread's amplitudes in its own
// CTA (the thread's top c index bits are its rank): shared-memory accesses
// and a CTA barrier.  A stage with a register bit among the top c reads and
// writes other CTAs' slices through distributed shared memory
// (ld / st.shared::cluster), with cluster barriers before and after it.

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Barrier over every thread of the cluster; orders the shared-memory
// accesses (local and distributed) before it against those after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void ld_cluster(uint32_t a, double2& v) {
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
}
__device__ __forceinline__ void ld_cluster(uint32_t a, float2& v) {
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, const double2& v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, const float2& v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}

// This CTA's slice of a cluster tile, addressed by tile index (the rank
// bits, all equal to this CTA's in a local stage, are dropped).
template <class A>
struct SliceTile {
  typename A::Cplx* t;
  uint32_t mask;  // 2^(k-c) - 1
  __device__ __forceinline__ typename A::Cplx load(uint32_t l) const { return t[l & mask]; }
  __device__ __forceinline__ void store(uint32_t l, const typename A::Cplx& v) const { t[l & mask] = v; }
};

// The whole cluster tile: element l in the slice of rank l >> shift.
template <class A>
struct ClusterTile {
  uint32_t base;  // shared address of the slice (the same offset in every CTA)
  uint32_t shift;
  __device__ __forceinline__ typename A::Cplx load(uint32_t l) const {
    typename A::Cplx v;
    ld_cluster(cluster_map(base + (l & ((1u << shift) - 1u)) * uint32_t(sizeof(v)), l >> shift), v);
    return v;
  }
  __device__ __forceinline__ void store(uint32_t l, const typename A::Cplx& v) const {
    st_cluster(cluster_map(base + (l & ((1u << shift) - 1u)) * uint32_t(sizeof(v)), l >> shift), v);
  }
};

// Shared-memory bytes of a cluster launch: the slice, chunk offsets, op
// list, stage list.
template <class A>
__host__ __device__ inline size_t cluster_smem_bytes(int k, int c, int L, int nops, int nstages) {
  return sizeof(typename A::Cplx) * (size_t(1) << (k - c)) + sizeof(int64_t) * (size_t(1) << (k - L)) +
         sizeof(FOp) * size_t(nops) + sizeof(FStage) * size_t(nstages);
}

// One pass over a single-tile register (P.ntiles == 1) on a cluster of C
// CTAs of 2^(k-R)/C threads.  Plain arithmetic only (float2 / double2).
template <class A, int R, int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kFusedThreads)
    k_fused_cluster(typename A::Store* __restrict__ g, const __grid_constant__ FPass P,
                    const FOp* __restrict__ ops, const FStage* __restrict__ stages) {
  using Cplx = typename A::Cplx;
  constexpr uint32_t c = C == 2 ? 1 : C == 4 ? 2 : 3;
  static_assert(C == 2 || C == 4 || C == 8, "cluster of 2, 4 or 8 CTAs");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = P.k, L = P.L;
  const uint32_t ks = uint32_t(k) - c;  // index bits of a slice
  PassSmem<A> m;
  m.tile = reinterpret_cast<Cplx*>(smem_raw);
  m.choff = reinterpret_cast<int64_t*>(smem_raw + sizeof(Cplx) * (size_t(1) << ks));
  m.ops = reinterpret_cast<FOp*>(m.choff + (1 << (k - L)));
  m.st = reinterpret_cast<FStage*>(m.ops + P.op_count);
  load_pass<A>(P, ops, stages, m);
  __syncthreads();
  const uint32_t rank = cluster_rank();
  const uint32_t nslice = 1u << ks, l0 = rank << ks;
  const uint32_t lmask_low = (1u << L) - 1u;
  // this CTA's slice from HBM (the register is one tile: base 0)
  if constexpr (sizeof(typename A::Store) == 8) {
    const float4* g4 = reinterpret_cast<const float4*>(g);
    float4* t4 = reinterpret_cast<float4*>(m.tile);
    for (uint32_t e = threadIdx.x; e < nslice / 2; e += blockDim.x) {
      const uint32_t l = l0 + 2 * e;
      t4[e] = g4[(m.choff[l >> L] + (l & lmask_low)) >> 1];
    }
  } else {
    for (uint32_t o = threadIdx.x; o < nslice; o += blockDim.x) {
      const uint32_t l = l0 + o;
      m.tile[o] = A::from_store(g[m.choff[l >> L] + (l & lmask_low)]);
    }
  }
  const SliceTile<A> slice{m.tile, nslice - 1u};
  const ClusterTile<A> whole{static_cast<uint32_t>(__cvta_generic_to_shared(m.tile)), ks};
  const uint32_t tidx = rank * blockDim.x + threadIdx.x;
  const int nst = P.stage_end - P.stage_begin;
  auto distributed = [&](int s) {
    bool d = false;
#pragma unroll
    for (int i = 0; i < R; ++i) d = d || m.st[s].pbits[i] >= ks;
    return d;
  };
  bool cur = nst > 0 && distributed(0);
  if (cur) cluster_sync();
  else __syncthreads();
  for (int s = 0; s < nst; ++s) {
    if (cur) run_stage<A, R>(whole, m.st[s], m.ops, tidx, 0);
    else run_stage<A, R>(slice, m.st[s], m.ops, tidx, 0);
    const bool next = s + 1 < nst && distributed(s + 1);
    if (cur || next) cluster_sync();  // other CTAs' slices read or written on either side
    else __syncthreads();
    cur = next;
  }
  // this CTA's slice back to HBM
  if constexpr (sizeof(typename A::Store) == 8) {
    float4* g4 = reinterpret_cast<float4*>(g);
    const float4* t4 = reinterpret_cast<const float4*>(m.tile);
    for (uint32_t e = threadIdx.x; e < nslice / 2; e += blockDim.x) {
      const uint32_t l = l0 + 2 * e;
      g4[(m.choff[l >> L] + (l & lmask_low)) >> 1] = t4[e];
    }
  } else {
    for (uint32_t o = threadIdx.x; o < nslice; o += blockDim.x) {
      const uint32_t l = l0 + o;
      g[m.choff[l >> L] + (l & lmask_low)] = A::to_store(m.tile[o]);
    }
  }
  cluster_sync();  // no CTA leaves while another could still address its slice
}

// Consecutive work items a CTA of the batched kernel takes at a time.
constexpr int kBatchChunk = 8;

// Batched: the work items of one wave (tiles of passes of many registers,
// each pass with its own register pointer).  Shared memory is laid out for
// the largest tile (kmax, Lmin) and op list (opmax) of the wave.
template <class A, int R>
__global__ void __launch_bounds__(kFusedThreads, fused_ctas_per_sm(R))
    k_fused_batch(const BItem* __restrict__ items, int nitems, const FPass* __restrict__ passes,
                  const FOp* __restrict__ ops, const FStage* __restrict__ stages, int kmax, int Lmin,
                  int opmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // The current pass's descriptor lives in shared memory (uniform per CTA;
  // its qubit list is indexed at run time, which in registers would force
  // the whole descriptor onto the stack).
  __shared__ FPass sP;
  PassSmem<A> m = pass_smem<A>(smem_raw, kmax, Lmin, opmax);
  int cur = -1;
  // runs of kBatchChunk consecutive items per CTA (block-cyclic): the items
  // of one pass are consecutive, so a CTA reloads a pass's op list once per
  // run instead of once per item
  for (int c = blockIdx.x; c * kBatchChunk < nitems; c += gridDim.x)
  for (int i = c * kBatchChunk, iend = min(nitems, (c + 1) * kBatchChunk); i < iend; ++i) {
    const BItem it = items[i];
    if (it.pass != cur) {
      cur = it.pass;
      if (threadIdx.x < sizeof(FPass) / 8)
        reinterpret_cast<uint64_t*>(&sP)[threadIdx.x] =
            reinterpret_cast<const uint64_t*>(passes + cur)[threadIdx.x];
      __syncthreads();
      load_pass<A>(sP, ops, stages, m);
      __syncthreads();
    }
    process_tile<A, R, true>(static_cast<typename A::Store*>(sP.amps), sP, it.tile, m);
  }
}

// Persistent batched form: one launch runs every wave.  The items of all
// waves are listed in wave order (pass w of a register before pass w + 1)
// and CTAs claim runs of kBatchChunk consecutive items from a global ticket,
// so the runs are claimed in list order.  Before the first item of a pass,
// thread 0 waits until every tile of the register's previous pass is done
// (done[prev] == need).  A waited-on item has a smaller index than the
// waiting one, so it was claimed earlier by a CTA that is running and never
// waits on a later item: the lowest unfinished claimed item can always
// proceed, and the launch cannot deadlock.  Each wait is still bounded by
// the global timer (max_ns); when one runs out the CTA sets bit 2 of the
// status word and stops claiming, and CTAs waiting on its items run out in
// turn.  done[] and the ticket are zeroed before every launch.
struct BDep {
  int32_t prev;  // pass whose tiles must all be done first (-1: none)
  int32_t need;  // its tile count
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t batch_globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}

// True once *count reaches need; false after max_ns of the global timer, or
// as soon as another CTA has reported a wait that ran out (status bit 2).
__device__ __forceinline__ bool batch_wait_count(const int* count, int need, const unsigned* status,
                                                 uint64_t max_ns) {
  if (ld_acquire_gpu(count) >= need) return true;
  const uint64_t t0 = batch_globaltimer();
  for (;;) {
    __nanosleep(100);
    if (ld_acquire_gpu(count) >= need) return true;
    if ((ld_volatile_u32(status) & 4u) || batch_globaltimer() - t0 > max_ns) return false;
  }
}

template <class A, int R>
__global__ void __launch_bounds__(kFusedThreads, fused_ctas_per_sm(R))
    k_fused_batch_persist(const BItem* __restrict__ items, int nitems, const FPass* __restrict__ passes,
                          const FOp* __restrict__ ops, const FStage* __restrict__ stages,
                          const BDep* __restrict__ deps, int* done, unsigned* ticket, unsigned* status,
                          int kmax, int Lmin, int opmax, uint64_t max_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ FPass sP;
  __shared__ int s_chunk, s_ok;
  PassSmem<A> m = pass_smem<A>(smem_raw, kmax, Lmin, opmax);
  int cur = -1;
  for (;;) {
    // after a wait ran out anywhere, stop claiming (the launch ends soon)
    if (threadIdx.x == 0) s_chunk = (ld_volatile_u32(status) & 4u) ? 0x7FFFFFFF / kBatchChunk : int(atomicAdd(ticket, 1u));
    __syncthreads();
    const int c = s_chunk;
    __syncthreads();  // every thread has read s_chunk before it is claimed again
    if (int64_t(c) * kBatchChunk >= nitems) return;
    const int iend = min(nitems, (c + 1) * kBatchChunk);
    for (int i = c * kBatchChunk; i < iend; ++i) {
      const BItem it = items[i];
      if (it.pass != cur) {
        cur = it.pass;
        if (threadIdx.x == 0) {
          const BDep d = deps[cur];
          bool ok = d.prev < 0 || batch_wait_count(done + d.prev, d.need, status, max_ns);
          if (!ok) atomicOr(status, 4u);
          __threadfence();
          s_ok = ok;
        }
        if (threadIdx.x < sizeof(FPass) / 8)
          reinterpret_cast<uint64_t*>(&sP)[threadIdx.x] =
              reinterpret_cast<const uint64_t*>(passes + cur)[threadIdx.x];
        __syncthreads();
        if (!s_ok) return;  // every thread leaves together; nothing is in flight
        load_pass<A>(sP, ops, stages, m);
        __syncthreads();
      }
      process_tile<A, R, true, true>(static_cast<typename A::Store*>(sP.amps), sP, it.tile, m);
      // the tile's stores, then its count (process_tile ends with a barrier
      // after the stores; each thread fences its own)
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(done + cur, 1);
      }
    }
  }
}

}  // namespace qs
