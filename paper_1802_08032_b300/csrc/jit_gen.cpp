// Source generator of the runtime-compiled pass kernels (see jit.h).
//
// The generated kernel does what k_fused<A, R> does for one pass, with the
// pass's structure as compile-time constants:
//   * tile base: the tile index with a zero inserted at every tile qubit;
//   * tile load / store: the same coalesced accesses as the interpreter
//     (complex64: two amplitudes per 16-byte access), each thread's chunk
//     offset computed once, the per-access part a constant;
//   * stages: register positions, copy bits and the register amplitudes'
//     shared-memory offsets are constants; every operation is one call of
//     the interpreter's own helper with its kind, register bits and masks as
//     template arguments, in plan order; conditions on local or global bits
//     stay run-time tests of the thread's local index and the tile base.
// Host code only (no CUDA runtime calls): the CPU planner tests generate and
// compile these sources without a GPU.
#include <algorithm>
#include <cstdio>
#include <sstream>

#include "jit.h"
#include "runtime.h"

namespace qs {

namespace {

const char* arith_name(Arith a) {
  switch (a) {
    case Arith::F32: return "qs::PlainArith<float>";
    case Arith::F64: return "qs::PlainArith<double>";
    default: return "qs::DFArith";
  }
}

const char* store_name(Arith a) { return a == Arith::F32 ? "float2" : "double2"; }

size_t store_bytes(Arith a) { return a == Arith::F32 ? 8 : 16; }
size_t cplx_bytes(Arith a) { return a == Arith::F32 ? 8 : 16; }  // float2, double2, dfc2 (4 floats)

// register-bit pair of a pair slot: (0,1) (0,2) (0,3) (0,4) (1,2) (1,3) (1,4) (2,3) (2,4) (3,4)
void pair_of_slot(int slot, int& a, int& b) {
  static const int A_[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
  static const int B_[10] = {1, 2, 3, 4, 2, 3, 4, 3, 4, 4};
  a = A_[slot];
  b = B_[slot];
}

std::string hex32(uint32_t x) {
  char buf[16];
  std::snprintf(buf, sizeof buf, "0x%08Xu", x);
  return buf;
}

std::string hex64(uint64_t x) {
  char buf[32];
  std::snprintf(buf, sizeof buf, "0x%016llXull", static_cast<unsigned long long>(x));
  return buf;
}

// The statement applying one op (without its condition), or throws.
std::string op_statement(const FOp& op, int o, int R, const JitShape& sh) {
  const int fam = op.code / kCodeSlots, slot = op.code % kCodeSlots;
  const std::string ref = "P.o[" + std::to_string(o) + "]";
  const std::string AR = "A, " + std::to_string(R);
  const uint32_t all = R >= 5 ? 0xFFFFFFFFu : ((1u << (1 << R)) - 1u);
  // fn<A, R, targs..., slot>(v[, mask][, op])
  auto bit = [&](const char* fn, const std::string& targs, bool with_op = true,
                 const std::string& mask = "") {
    if (slot >= R) fail(QS_E_ARG, "jit: register bit beyond R");
    return std::string(fn) + "<" + AR + targs + std::to_string(slot) + ">(v" + (mask.empty() ? "" : ", " + mask) +
           (with_op ? ", " + ref : "") + ");";
  };
  auto pair_slot = [&](const char* fn) {
    if (slot > 9) fail(QS_E_ARG, "jit: pair slot beyond 9");
    int a, b;
    pair_of_slot(slot, a, b);
    if (b >= R) fail(QS_E_ARG, "jit: register pair beyond R");
    return std::string(fn) + "<" + AR + ", " + std::to_string(a) + ", " + std::to_string(b) + ">(v, " +
           ref + ");";
  };
  auto only0 = [&]() {
    if (slot != 0) fail(QS_E_ARG, "jit: unexpected slot");
  };
  auto side = [&](const char* kind, bool conj) {
    if (!(sh.arith == Arith::F64 && R == 4)) fail(QS_E_ARG, "jit: side-factor op outside FP64 R = 4");
    const int I = slot / 4, J = slot % 4;
    if (I >= 4 || J >= 4 || I == J) fail(QS_E_ARG, "jit: bad side-factor slot");
    return std::string("pair_side_on_bit<") + AR + ", " + kind + ", " + (conj ? "true" : "false") + ", " +
           std::to_string(I) + ", " + std::to_string(J) + ">(v, " + ref + ");";
  };
  const std::string rm = hex32(op.rmask);
  switch (fam) {
    case FC_GEN: return bit("pair_on_bit", ", PK_GEN, false, true, ", true, rm);
    case FC_GEN_C: return bit("pair_on_bit", ", PK_GEN, true, true, ", true, rm);
    case FC_H: return bit("pair_on_bit", ", PK_H, false, false, ", true, "0u");
    case FC_SX: return bit("pair_on_bit", ", PK_SX, false, false, ", true, "0u");
    case FC_SX_C: return bit("pair_on_bit", ", PK_SX, true, false, ", true, "0u");
    case FC_SY: return bit("pair_on_bit", ", PK_SY, false, false, ", true, "0u");
    case FC_X: return bit("pair_on_bit", ", PK_X, false, true, ", true, rm);
    case FC_PHASE_BIT: return bit("phase_on_bit", ", ");
    case FC_PHASE_ALL: only0(); return "phase_mask<" + AR + ", " + hex32(all) + ">(v, " + ref + ");";
    case FC_PHASE_MASK: only0(); return "phase_mask<" + AR + ", " + hex32(op.c.u[15] & all) + ">(v, " + ref + ");";
    case FC_SIGN: only0(); return "negate_mask<" + AR + ", " + hex32(op.c.u[15] & all) + ">(v);";
    case FC_DEPH: {
      only0();
      if (op.asrc > BS_GLOBAL || op.bsrc > BS_GLOBAL) fail(QS_E_ARG, "jit: bad bit source");
      return "deph_src<" + AR + ", " + std::to_string(op.asrc) + ", " + std::to_string(op.apos) + ", " +
             std::to_string(op.bsrc) + ", " + std::to_string(op.bpos) + ">(v, tl, (uint64_t)base, " + ref + ");";
    }
    case FC_DEPOL: return pair_slot("depol_on_bits");
    case FC_SCALE: only0(); return "phase_mask<" + AR + ", " + hex32(all) + ">(v, " + ref + ");";
    case FC_MULI_BIT: return bit("muli_on_bit", ", ", false);
    case FC_MULI_ALL: only0(); return "muli_mask<" + AR + ", " + hex32(all) + ">(v);";
    case FC_MULI_MASK: only0(); return "muli_mask<" + AR + ", " + hex32(op.c.u[15] & all) + ">(v);";
    case FC_SHEAR:
      if (slot >= R) fail(QS_E_ARG, "jit: register bit beyond R");
      return "shear_on_bit<" + AR + ", " + std::to_string(slot) + ", 0>(v, " + ref + ");";
    case FC_SHEAR2:
      if (slot >= R) fail(QS_E_ARG, "jit: register bit beyond R");
      return "shear_on_bit<" + AR + ", " + std::to_string(slot) + ", 1>(v, " + ref + ");";
    case FC_PHASEU_BIT: return bit("phaseu_on_bit", ", ");
    case FC_PHASEU_ALL: only0(); return "phaseu_mask<" + AR + ", " + hex32(all) + ">(v, " + ref + ");";
    case FC_DEPH_PAIR: return pair_slot("deph_on_bits");
    case FC_OFFPH: return pair_slot("offph_on_bits");
    case FC_H_SIDE: return side("PK_H", false);
    case FC_SX_SIDE: return side("PK_SX", false);
    case FC_SX_C_SIDE: return side("PK_SX", true);
    case FC_SY_SIDE: return side("PK_SY", false);
    default: break;
  }
  fail(QS_E_ARG, "jit: unknown op family " + std::to_string(fam));
}

// True when the set m of register amplitudes is not invariant under
// toggling register bit i (a sign flip on m does not commute with a pair
// update on bit i).
bool depends_on(uint32_t m, int i, int R) {
  if (i < 0 || i >= R) return true;
  uint32_t moved = 0;
  for (int j = 0; j < (1 << R); ++j)
    if ((m >> j) & 1u) moved |= 1u << (j ^ (1 << i));
  return moved != m;
}

}  // namespace

size_t jit_smem_bytes(const FPass& fp, const JitShape& sh) {
  const size_t tile = cplx_bytes(sh.arith) * (size_t(1) << fp.k);
  if (sh.copy == JitCopy::Bulk) return 2 * tile + 2 * sizeof(uint64_t);
  if (sh.copy == JitCopy::Async) return 2 * tile;
  return tile;
}

std::string jit_source(const FPass& fp, const FStage* st, const FOp* ops, const JitShape& sh) {
  const int R = sh.R, k = fp.k, L = fp.L;
  if (R < 1 || R > 5 || k < R || k > 20 || L < 1 || L > k) fail(QS_E_ARG, "jit: bad tile shape");
  if (fp.init) fail(QS_E_ARG, "jit: generated tiles are not supported");
  const int T = 1 << (k - R);
  const bool bulk = sh.copy == JitCopy::Bulk, async = sh.copy == JitCopy::Async;
  const bool pipelined = bulk || async;  // two buffers, tiles kept in the storage format
  const bool pack2 = store_bytes(sh.arith) == 8;  // complex64: two amplitudes per access
  const int span_log = pack2 ? (k - R + 1) : (k - R);  // amplitudes one round of accesses covers (log2)
  if (!bulk && span_log < L) fail(QS_E_ARG, "jit: access round narrower than a chunk");
  if (bulk && (R < L || (size_t(1) << L) * store_bytes(sh.arith) % 16 != 0))
    fail(QS_E_ARG, "jit: chunks unsuited to bulk copies");
  const int depth = pack2 ? (1 << (R - 1)) : (1 << R);
  const int cbits = span_log - L;  // chunk-index bits taken from the thread index
  auto deposit = [&](uint64_t c) {  // chunk index -> offset (bit i at tile qubit L + i)
    uint64_t off = 0;
    for (int i = 0; c >> i; ++i)
      if ((c >> i) & 1u) off |= uint64_t(1) << fp.q[L + i];
    return off;
  };
  // Shared-memory swizzle: amplitude l of the tile lives at sw(l) = l ^ h(l),
  // h XOR-ing the amplitude's slot within a 128-byte row with a fold of the
  // index bits above the row, so that a warp whose 32 threads differ only
  // in high local positions (a stage whose register bits hold the low ones)
  // spreads over the banks instead of hitting one.  h is linear over XOR, so
  // sw(tl | c) = sw(tl) ^ sw(c) for disjoint bits: one per-thread term and
  // one constant per access.  Complex64 keeps amplitude pairs (2i, 2i + 1)
  // together (16-byte accesses).  Off for bulk copies (whole chunks).
  const bool swz = sh.swizzle && !bulk;
  auto hsw = [&](uint64_t x) -> uint64_t {
    if (!swz) return 0;
    if (pack2) return (((x >> 4) ^ (x >> 7) ^ (x >> 10)) & 7u) << 1;
    return ((x >> 3) ^ (x >> 6) ^ (x >> 9)) & 7u;
  };
  auto sw = [&](uint64_t x) { return x ^ hsw(x); };
  auto hsw_expr = [&](const std::string& v) -> std::string {
    if (!swz) return "0u";
    if (pack2) return "(((((" + v + ") >> 4) ^ ((" + v + ") >> 7) ^ ((" + v + ") >> 10)) & 7u) << 1)";
    return "((((" + v + ") >> 3) ^ ((" + v + ") >> 6) ^ ((" + v + ") >> 9)) & 7u)";
  };
  const int nstage = fp.stage_end - fp.stage_begin;
  // the last stage stores to HBM itself (no shared-memory round trip and
  // store phase); the bulk form stores whole chunks from shared memory
  const bool direct_last = sh.direct_store && !bulk && nstage > 0;
  std::ostringstream s;
  s << "// fused pass: k " << k << " L " << L << " R " << R << " ops " << fp.op_count << " stages " << nstage
    << (bulk ? " (bulk-copy pipeline)" : async ? " (async-copy pipeline)" : "") << "\n";
  s << "#ifdef __CUDACC_RTC__\n"
       "typedef signed char int8_t; typedef unsigned char uint8_t; typedef short int16_t;\n"
       "typedef unsigned short uint16_t; typedef int int32_t; typedef unsigned int uint32_t;\n"
       "typedef long long int64_t; typedef unsigned long long uint64_t;\n"
       "#endif\n"
       "#include \"fused_arith.cuh\"\n";
  if (pipelined) s << "#include \"mbarrier.cuh\"\n";
  s << "namespace qs { struct JitOps { FOp o[" << (fp.op_count > 0 ? fp.op_count : 1) << "]; }; }\n"
    << "using namespace qs;\n"
    << "extern \"C\" __global__ void __launch_bounds__(" << T << ", " << sh.ctas << ")\n"
    << "qs_pass(" << store_name(sh.arith) << "* __restrict__ g, long long ntiles,\n"
    << (bulk ? "        unsigned* __restrict__ status,\n" : "")
    << "        const __grid_constant__ qs::JitOps P) {\n"
    << "  using A = " << arith_name(sh.arith) << ";\n"
    << "  using Cplx = A::Cplx;\n"
    << "  using Store = A::Store;\n"
    << "  extern __shared__ __align__(128) unsigned char smem_raw[];\n"
    << "  const uint32_t tid = threadIdx.x;\n";
  // tile base: the tile index with a zero inserted at every tile qubit
  s << "  auto tile_base = [](int64_t t) {\n    int64_t b = t << " << L << ";\n";
  for (int i = L; i < k; ++i) {
    const int p = fp.q[i];
    s << "    b = ((b >> " << p << ") << " << (p + 1) << ") | (b & " << hex64((uint64_t(1) << p) - 1) << ");\n";
  }
  s << "    return b;\n  };\n";
  const size_t chunk_bytes = (size_t(1) << L) * store_bytes(sh.arith);
  const size_t tile_store_bytes = (size_t(1) << k) * store_bytes(sh.arith);
  if (!bulk) {
    // this thread's part of the tile offset of its coalesced accesses
    s << "  const uint32_t lt = " << (pack2 ? "2u * tid" : "tid") << ";\n"
      << "  int64_t toff = int64_t(lt & " << hex32((1u << L) - 1u) << ");\n";
    for (int i = 0; i < cbits; ++i)
      s << "  toff |= int64_t((lt >> " << (L + i) << ") & 1u) << " << int(fp.q[L + i]) << ";\n";
    // shared-memory index of its accesses (amplitude units; swizzled)
    s << "  const uint32_t slt = lt ^ " << hsw_expr("lt") << ";\n";
  }
  // (global offset, shared index) of this thread's u-th coalesced access
  auto acc_goff = [&](int u) { return hex64(deposit(uint64_t(u) << cbits)); };
  if (bulk) {
    // Bulk (TMA) copies: the tile is 2^(k-L) contiguous chunks of 2^L
    // amplitudes; thread t copies chunks t + T u (u < 2^(R-L)) in and out, so
    // each thread only ever overwrites chunks whose stores it issued itself.
    s << "  Cplx* const buf0 = reinterpret_cast<Cplx*>(smem_raw);\n"
      << "  Cplx* const buf1 = buf0 + " << (1 << k) << ";\n"
      << "  uint64_t* const bar = reinterpret_cast<uint64_t*>(buf0 + " << (2 << k) << ");\n"
      << "  int64_t coff = 0;  // this thread's chunk offset\n";
    for (int i = 0; i < k - R; ++i)
      s << "  coff |= int64_t((tid >> " << i << ") & 1u) << " << int(fp.q[L + i]) << ";\n";
    const int per = 1 << (R - L);
    s << "  auto issue_load = [&](int64_t b, Cplx* dst, uint64_t* br) {\n";
    for (int u = 0; u < per; ++u) {
      const uint64_t cu = uint64_t(u) << (k - R);
      s << "    mb::bulk_load(reinterpret_cast<Store*>(dst) + ((tid + " << cu << "u) << " << L << "), g + b + coff + "
        << hex64(deposit(cu)) << ", " << chunk_bytes << "u, br);\n";
    }
    s << "  };\n  auto issue_store = [&](int64_t b, Cplx* src) {\n";
    for (int u = 0; u < per; ++u) {
      const uint64_t cu = uint64_t(u) << (k - R);
      s << "    mb::bulk_store(g + b + coff + " << hex64(deposit(cu)) << ", reinterpret_cast<Store*>(src) + ((tid + "
        << cu << "u) << " << L << "), " << chunk_bytes << "u);\n";
    }
    s << "    mb::bulk_commit();\n  };\n";
    // thread 0 announces the bytes before anyone's copy can complete on the
    // barrier (the barrier after it orders the copies behind it)
    s << "  if (tid == 0) {\n    mb::init(&bar[0], 1);\n    mb::init(&bar[1], 1);\n    mb::fence_init();\n  }\n"
      << "  __syncthreads();\n"
      << "  int64_t tau = blockIdx.x;\n"
      << "  if (tau < ntiles) {\n"
      << "    if (tid == 0) mb::arrive_expect_tx(&bar[0], " << tile_store_bytes << "u);\n"
      << "    __syncthreads();\n"
      << "    issue_load(tile_base(tau), buf0, &bar[0]);\n"
      << "  }\n"
      << "  uint32_t parity = 0;  // bit i: parity of buffer i's next phase\n"
      << "  bool pend[2] = {tau < ntiles, false};\n"
      << "  bool ok = true;\n"
      << "  for (int it = 0; tau < ntiles; ++it, tau += gridDim.x) {\n"
      << "    const int cur = it & 1;\n"
      << "    Cplx* const tile = cur ? buf1 : buf0;\n"
      << "    const int64_t base = tile_base(tau);\n"
      << "    const bool more = tau + int64_t(gridDim.x) < ntiles;\n"
      << "    if (more) {\n"
      << "      mb::bulk_wait_read();  // this thread's stores from the other buffer have read it\n"
      << "      if (tid == 0) mb::arrive_expect_tx(&bar[cur ^ 1], " << tile_store_bytes << "u);\n"
      << "      __syncthreads();\n"
      << "      issue_load(tile_base(tau + gridDim.x), cur ? buf0 : buf1, &bar[cur ^ 1]);\n"
      << "    }\n"
      << "    pend[cur ^ 1] = more;\n"
      << "    const bool got = mb::wait(&bar[cur], (parity >> cur) & 1u);\n"
      << "    if (!__syncthreads_and(got)) {\n      ok = false;\n      break;\n    }\n"
      << "    parity ^= 1u << cur;\n"
      << "    pend[cur] = false;\n";
  } else if (async) {
    // Async copies (cp.async, 16 bytes a thread): the same coalesced
    // accesses as the plain load, into the other buffer, one group per tile.
    s << "  Cplx* const buf0 = reinterpret_cast<Cplx*>(smem_raw);\n"
      << "  Cplx* const buf1 = buf0 + " << (1 << k) << ";\n"
      << "  auto issue_load = [&](int64_t b, Cplx* dst) {\n"
      << "    const int64_t gb = b + toff;\n";
    for (int u = 0; u < depth; ++u) {
      if (pack2)
        s << "    mb::async_copy16(reinterpret_cast<float4*>(dst) + ((slt ^ " << hex32(uint32_t(sw(uint64_t(2 * u * T))))
          << ") >> 1), reinterpret_cast<const float4*>(g) + ((gb + " << acc_goff(u) << ") >> 1));\n";
      else
        s << "    mb::async_copy16(reinterpret_cast<Store*>(dst) + (slt ^ " << hex32(uint32_t(sw(uint64_t(u * T))))
          << "), g + gb + " << acc_goff(u) << ");\n";
    }
    s << "    asm volatile(\"cp.async.commit_group;\" ::: \"memory\");\n  };\n"
      << "  int64_t tau = blockIdx.x;\n"
      << "  if (tau < ntiles) issue_load(tile_base(tau), buf0);\n"
      << "  for (int it = 0; tau < ntiles; ++it, tau += gridDim.x) {\n"
      << "    const int cur = it & 1;\n"
      << "    Cplx* const tile = cur ? buf1 : buf0;\n"
      << "    const int64_t base = tile_base(tau);\n"
      << "    if (tau + int64_t(gridDim.x) < ntiles) {\n"
      << "      issue_load(tile_base(tau + gridDim.x), cur ? buf0 : buf1);\n"
      << "      asm volatile(\"cp.async.wait_group 1;\" ::: \"memory\");\n"
      << "    } else {\n"
      << "      asm volatile(\"cp.async.wait_group 0;\" ::: \"memory\");\n"
      << "    }\n"
      << "    __syncthreads();\n";
  } else {
    s << "  Cplx* __restrict__ tile = reinterpret_cast<Cplx*>(smem_raw);\n"
      << "  for (int64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {\n"
      << "    const int64_t base = tile_base(tau);\n";
    // tile load: all accesses of the round in flight, then into shared memory
    if (pack2) {
      s << "    {\n      const float4* __restrict__ g4 = reinterpret_cast<const float4*>(g);\n"
        << "      float4* t4 = reinterpret_cast<float4*>(tile);\n"
        << "      const int64_t gb = base + toff;\n";
      for (int u = 0; u < depth; ++u)
        s << "      const float4 ld" << u << " = g4[(gb + " << acc_goff(u) << ") >> 1];\n";
      for (int u = 0; u < depth; ++u)
        s << "      t4[(slt ^ " << hex32(uint32_t(sw(uint64_t(2 * u * T)))) << ") >> 1] = ld" << u << ";\n";
      s << "    }\n";
    } else {
      s << "    {\n      const int64_t gb = base + toff;\n";
      for (int u = 0; u < depth; ++u) s << "      const double2 ld" << u << " = g[gb + " << acc_goff(u) << "];\n";
      for (int u = 0; u < depth; ++u)
        s << "      tile[slt ^ " << hex32(uint32_t(sw(uint64_t(u * T)))) << "] = A::from_store(ld" << u << ");\n";
      s << "    }\n";
    }
    s << "    __syncthreads();\n";
  }
  for (int si = fp.stage_begin; si < fp.stage_end; ++si) {
    const FStage& S = st[si];
    // with a copy pipeline the tile arrives and leaves in the storage
    // format: the first stage converts on reading, the last on writing
    const bool first_io = pipelined && si == fp.stage_begin;
    const bool last_io = pipelined && si == fp.stage_end - 1;
    uint32_t poff[8] = {}, cpm = 0;
    for (int i = 0; i < R; ++i) {
      if (S.pbits[i] >= k) fail(QS_E_ARG, "jit: register position outside the tile");
      poff[i] = 1u << S.pbits[i];
      if ((S.copy >> i) & 1u) cpm |= poff[i];
    }
    // complex64 with register bit 0 at local position 0: amplitudes j and
    // j + 1 are neighbours in shared memory, one 16-byte access
    const bool vec2 = pack2 && S.pbits[0] == 0 && !(cpm & 1u);
    s << "    {\n      uint32_t tl = tid;\n";
    for (int i = 0; i < R; ++i) {
      const int p = S.pbits[i];
      s << "      tl = ((tl >> " << p << ") << " << (p + 1) << ") | (tl & " << hex32((1u << p) - 1u) << ");\n";
    }
    s << "      const uint32_t stl = tl ^ " << hsw_expr("tl") << ";\n";
    s << "      Cplx v[" << (1 << R) << "];\n";
    std::vector<uint32_t> off(size_t(1) << R);
    for (int j = 0; j < (1 << R); ++j) {
      uint32_t o = 0;
      for (int i = 0; i < R; ++i)
        if (j & (1 << i)) o |= poff[i];
      off[size_t(j)] = o;
    }
    for (int j = 0; j < (1 << R); ++j) {
      const uint32_t o = off[size_t(j)];
      if (vec2) {
        if (j & 1) continue;
        s << "      {\n        const float4 w = *reinterpret_cast<const float4*>(tile + (stl ^ "
          << hex32(uint32_t(sw(o & ~cpm))) << "));\n        v[" << j << "] = make_float2(w.x, w.y);\n        v[" << j + 1
          << "] = make_float2(w.z, w.w);\n      }\n";
      } else if (first_io) {
        s << "      v[" << j << "] = A::from_store(reinterpret_cast<const Store*>(tile)[stl ^ "
          << hex32(uint32_t(sw(o & ~cpm))) << "]);\n";
      } else {
        s << "      v[" << j << "] = tile[stl ^ " << hex32(uint32_t(sw(o & ~cpm))) << "];\n";
      }
    }
    // Sign flips (CZ, multi-controlled phase flips) are kept pending, as
    // the interpreter keeps them: an unconditional compile-time mask, and
    // per-thread booleans for flips conditioned on local or global bits
    // (one per distinct mask, merged by XOR); each is applied just before
    // the first op it does not commute with, or at the end of the stage.
    // Negation is exact and commutes exactly with what it is moved past, so
    // the results are those of applying it where it occurs.
    uint32_t unc = 0;
    std::vector<std::pair<uint32_t, std::string>> pend;  // (mask, bool variable)
    int nflag = 0;
    const std::string AR = "A, " + std::to_string(R);
    auto apply_unc = [&]() {
      if (unc) s << "      negate_mask<" << AR << ", " << hex32(unc) << ">(v);\n";
      unc = 0;
    };
    auto apply_pend = [&](size_t i) {
      s << "      if (" << pend[i].second << ") negate_mask<" << AR << ", " << hex32(pend[i].first) << ">(v);\n";
    };
    for (int o = S.op_begin; o < S.op_end; ++o) {
      if (o < 0 || o >= fp.op_count) fail(QS_E_ARG, "jit: stage op range outside the pass");
      const FOp& op = ops[fp.op_begin + o];
      std::string cond;
      if ((op.flags & FF_COND) && (op.lmask || op.gmask)) {
        if (op.lmask) cond += "(tl & " + hex32(op.lmask) + ") == " + hex32(op.lmask);
        if (op.lmask && op.gmask) cond += " && ";
        if (op.gmask) cond += "((uint64_t)base & " + hex64(op.gmask) + ") == " + hex64(op.gmask);
      }
      if (op.code == FC_SIGN * kCodeSlots) {
        const uint32_t m = op.c.u[15] & (R >= 5 ? 0xFFFFFFFFu : ((1u << (1 << R)) - 1u));
        if (!m) continue;
        if (cond.empty()) {
          unc ^= m;
          continue;
        }
        size_t i = 0;
        while (i < pend.size() && pend[i].first != m) ++i;
        if (i == pend.size()) {
          const std::string var = "f" + std::to_string(nflag++);
          s << "      bool " << var << " = " << cond << ";\n";
          pend.emplace_back(m, var);
        } else {
          s << "      " << pend[i].second << " ^= (" << cond << ");\n";
        }
        continue;
      }
      if (op.flags & FF_FLIP) {
        const int b0 = op.i0, b1 = (op.flags & FF_TWO) ? op.i1 : -1;
        auto dep = [&](uint32_t m) {
          return depends_on(m, b0, R) || (b1 >= 0 && depends_on(m, b1, R));
        };
        if (unc && dep(unc)) apply_unc();
        for (size_t i = 0; i < pend.size();) {
          if (dep(pend[i].first)) {
            apply_pend(i);
            pend.erase(pend.begin() + long(i));
          } else {
            ++i;
          }
        }
      }
      const std::string stmt = op_statement(op, o, R, sh);
      if (!cond.empty()) s << "      if (" << cond << ") " << stmt << "\n";
      else s << "      " << stmt << "\n";
    }
    apply_unc();
    for (size_t i = 0; i < pend.size(); ++i) apply_pend(i);
    const bool direct = direct_last && si == fp.stage_end - 1;
    if (direct) {
      // The last stage writes its amplitudes straight to HBM: local index
      // tl | off maps to the global offset D(tl) + D(off) (the low L bits
      // in place, bit i >= L at tile qubit q[i]); a warp's stores of one
      // register amplitude cover whole sectors once its other amplitudes
      // are written, which L2 merges before they reach DRAM.
      auto dmap = [&](uint32_t l) {
        uint64_t d = l & ((1u << L) - 1u);
        for (int b = L; b < k; ++b)
          if ((l >> b) & 1u) d |= uint64_t(1) << fp.q[b];
        return d;
      };
      s << "      int64_t dtl = int64_t(tl & " << hex32((1u << L) - 1u) << ");\n";
      for (int b = L; b < k; ++b) {
        bool reg = false;
        for (int i = 0; i < R; ++i) reg = reg || S.pbits[i] == b;
        if (!reg) s << "      dtl |= int64_t((tl >> " << b << ") & 1u) << " << int(fp.q[b]) << ";\n";
      }
      s << "      Store* const gt = g + base + dtl;\n";
      for (int j = 0; j < (1 << R); ++j) {
        const uint64_t d = dmap(off[size_t(j)]);
        if (vec2) {
          if (j & 1) continue;
          s << "      *reinterpret_cast<float4*>(gt + " << hex64(d) << ") = make_float4(v[" << j << "].x, v[" << j
            << "].y, v[" << j + 1 << "].x, v[" << j + 1 << "].y);\n";
        } else {
          s << "      gt[" << hex64(d) << "] = A::to_store(v[" << j << "]);\n";
        }
      }
      s << "    }\n    __syncthreads();\n";
      continue;
    }
    // (each thread writes exactly the slots it read: converting in place
    // needs no barrier)
    for (int j = 0; j < (1 << R); ++j) {
      const uint32_t o = off[size_t(j)];
      if (vec2) {
        if (j & 1) continue;
        s << "      *reinterpret_cast<float4*>(tile + (stl ^ " << hex32(uint32_t(sw(o))) << ")) = make_float4(v[" << j << "].x, v["
          << j << "].y, v[" << j + 1 << "].x, v[" << j + 1 << "].y);\n";
      } else if (last_io) {
        s << "      reinterpret_cast<Store*>(tile)[stl ^ " << hex32(uint32_t(sw(o))) << "] = A::to_store(v[" << j << "]);\n";
      } else {
        s << "      tile[stl ^ " << hex32(uint32_t(sw(o))) << "] = v[" << j << "];\n";
      }
    }
    s << "    }\n    __syncthreads();\n";
  }
  if (bulk) {
    s << "    mb::fence_proxy_async();\n"
      << "    __syncthreads();\n"
      << "    issue_store(base, tile);\n"
      << "  }\n"
      << "  if (!ok) {\n"
      << "    // a copy did not arrive within the bound: report it, and wait (bounded)\n"
      << "    // for copies still in flight into this CTA's shared memory\n"
      << "    if (tid == 0) atomicOr(status, 2u);\n"
      << "    for (int i = 0; i < 2; ++i)\n"
      << "      if (pend[i]) (void)mb::wait(&bar[i], (parity >> i) & 1u);\n"
      << "  }\n"
      << "  mb::bulk_wait();\n"
      << "}\n";
    return s.str();
  }
  if (direct_last) {
    s << "  }\n}\n";
    return s.str();
  }
  s << "    // tile store\n";
  if (pack2) {
    s << "    {\n      float4* __restrict__ g4 = reinterpret_cast<float4*>(g);\n"
      << "      const float4* t4 = reinterpret_cast<const float4*>(tile);\n"
      << "      const int64_t gb = base + toff;\n";
    for (int u = 0; u < depth; ++u)
      s << "      g4[(gb + " << acc_goff(u) << ") >> 1] = t4[(slt ^ " << hex32(uint32_t(sw(uint64_t(2 * u * T))))
        << ") >> 1];\n";
    s << "    }\n";
  } else {
    s << "    {\n      const int64_t gb = base + toff;\n";
    for (int u = 0; u < depth; ++u) {
      if (async)  // already in the storage format
        s << "      g[gb + " << acc_goff(u) << "] = reinterpret_cast<const Store*>(tile)[slt ^ "
          << hex32(uint32_t(sw(uint64_t(u * T)))) << "];\n";
      else
        s << "      g[gb + " << acc_goff(u) << "] = A::to_store(tile[slt ^ " << hex32(uint32_t(sw(uint64_t(u * T))))
          << "]);\n";
    }
    s << "    }\n";
  }
  s << "    __syncthreads();\n  }\n}\n";
  return s.str();
}

}  // namespace qs
