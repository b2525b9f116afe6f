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

}  // namespace

size_t jit_smem_bytes(const FPass& fp, Arith a) { return cplx_bytes(a) * (size_t(1) << fp.k); }

std::string jit_source(const FPass& fp, const FStage* st, const FOp* ops, const JitShape& sh) {
  const int R = sh.R, k = fp.k, L = fp.L;
  if (R < 1 || R > 5 || k < R || k > 20 || L < 1 || L > k) fail(QS_E_ARG, "jit: bad tile shape");
  if (fp.init) fail(QS_E_ARG, "jit: generated tiles are not supported");
  const int T = 1 << (k - R);
  const bool pack2 = store_bytes(sh.arith) == 8;  // complex64: two amplitudes per access
  const int span_log = pack2 ? (k - R + 1) : (k - R);  // amplitudes one round of accesses covers (log2)
  if (span_log < L) fail(QS_E_ARG, "jit: access round narrower than a chunk");
  const int depth = pack2 ? (1 << (R - 1)) : (1 << R);
  const int cbits = span_log - L;  // chunk-index bits taken from the thread index
  auto deposit = [&](uint64_t c) {  // chunk index -> offset (bit i at tile qubit L + i)
    uint64_t off = 0;
    for (int i = 0; c >> i; ++i)
      if ((c >> i) & 1u) off |= uint64_t(1) << fp.q[L + i];
    return off;
  };
  std::ostringstream s;
  s << "// fused pass: k " << k << " L " << L << " R " << R << " ops " << fp.op_count << " stages "
    << (fp.stage_end - fp.stage_begin) << "\n";
  s << "#ifdef __CUDACC_RTC__\n"
       "typedef signed char int8_t; typedef unsigned char uint8_t; typedef short int16_t;\n"
       "typedef unsigned short uint16_t; typedef int int32_t; typedef unsigned int uint32_t;\n"
       "typedef long long int64_t; typedef unsigned long long uint64_t;\n"
       "#endif\n"
       "#include \"fused_arith.cuh\"\n"
       "namespace qs { struct JitOps { FOp o["
    << (fp.op_count > 0 ? fp.op_count : 1) << "]; }; }\n"
    << "using namespace qs;\n"
    << "extern \"C\" __global__ void __launch_bounds__(" << T << ", " << sh.ctas << ")\n"
    << "qs_pass(" << store_name(sh.arith) << "* __restrict__ g, long long ntiles,\n"
    << "        const __grid_constant__ qs::JitOps P) {\n"
    << "  using A = " << arith_name(sh.arith) << ";\n"
    << "  using Cplx = A::Cplx;\n"
    << "  extern __shared__ __align__(16) unsigned char smem_raw[];\n"
    << "  Cplx* __restrict__ tile = reinterpret_cast<Cplx*>(smem_raw);\n"
    << "  const uint32_t tid = threadIdx.x;\n";
  // this thread's part of the tile offset of its accesses
  s << "  const uint32_t lt = " << (pack2 ? "2u * tid" : "tid") << ";\n"
    << "  int64_t toff = int64_t(lt & " << hex32((1u << L) - 1u) << ");\n";
  for (int i = 0; i < cbits; ++i)
    s << "  toff |= int64_t((lt >> " << (L + i) << ") & 1u) << " << int(fp.q[L + i]) << ";\n";
  s << "  for (int64_t tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {\n"
    << "    int64_t base = tau << " << L << ";\n";
  for (int i = L; i < k; ++i) {
    const int p = fp.q[i];
    s << "    base = ((base >> " << p << ") << " << (p + 1) << ") | (base & " << hex64((uint64_t(1) << p) - 1)
      << ");\n";
  }
  // tile load: all accesses of the round in flight, then into shared memory
  if (pack2) {
    s << "    {\n      const float4* __restrict__ g4 = reinterpret_cast<const float4*>(g);\n"
      << "      float4* t4 = reinterpret_cast<float4*>(tile);\n"
      << "      const int64_t gb = base + toff;\n";
    for (int u = 0; u < depth; ++u)
      s << "      const float4 ld" << u << " = g4[(gb + " << hex64(deposit(uint64_t(u) << cbits)) << ") >> 1];\n";
    for (int u = 0; u < depth; ++u) s << "      t4[tid + " << u * T << "u] = ld" << u << ";\n";
    s << "    }\n";
  } else {
    s << "    {\n      const int64_t gb = base + toff;\n";
    for (int u = 0; u < depth; ++u)
      s << "      const double2 ld" << u << " = g[gb + " << hex64(deposit(uint64_t(u) << cbits)) << "];\n";
    for (int u = 0; u < depth; ++u) s << "      tile[tid + " << u * T << "u] = A::from_store(ld" << u << ");\n";
    s << "    }\n";
  }
  s << "    __syncthreads();\n";
  for (int si = fp.stage_begin; si < fp.stage_end; ++si) {
    const FStage& S = st[si];
    uint32_t poff[8] = {}, cpm = 0;
    for (int i = 0; i < R; ++i) {
      if (S.pbits[i] >= k) fail(QS_E_ARG, "jit: register position outside the tile");
      poff[i] = 1u << S.pbits[i];
      if ((S.copy >> i) & 1u) cpm |= poff[i];
    }
    s << "    {\n      uint32_t tl = tid;\n";
    for (int i = 0; i < R; ++i) {
      const int p = S.pbits[i];
      s << "      tl = ((tl >> " << p << ") << " << (p + 1) << ") | (tl & " << hex32((1u << p) - 1u) << ");\n";
    }
    s << "      Cplx v[" << (1 << R) << "];\n";
    std::vector<uint32_t> off(size_t(1) << R);
    for (int j = 0; j < (1 << R); ++j) {
      uint32_t o = 0;
      for (int i = 0; i < R; ++i)
        if (j & (1 << i)) o |= poff[i];
      off[size_t(j)] = o;
      s << "      v[" << j << "] = tile[tl | " << hex32(o & ~cpm) << "];\n";
    }
    for (int o = S.op_begin; o < S.op_end; ++o) {
      if (o < 0 || o >= fp.op_count) fail(QS_E_ARG, "jit: stage op range outside the pass");
      const FOp& op = ops[fp.op_begin + o];
      const std::string stmt = op_statement(op, o, R, sh);
      if ((op.flags & FF_COND) && (op.lmask || op.gmask)) {
        s << "      if (";
        if (op.lmask) s << "(tl & " << hex32(op.lmask) << ") == " << hex32(op.lmask);
        if (op.lmask && op.gmask) s << " && ";
        if (op.gmask) s << "((uint64_t)base & " << hex64(op.gmask) << ") == " << hex64(op.gmask);
        s << ") " << stmt << "\n";
      } else {
        s << "      " << stmt << "\n";
      }
    }
    for (int j = 0; j < (1 << R); ++j) s << "      tile[tl | " << hex32(off[size_t(j)]) << "] = v[" << j << "];\n";
    s << "    }\n    __syncthreads();\n";
  }
  // tile store
  if (pack2) {
    s << "    {\n      float4* __restrict__ g4 = reinterpret_cast<float4*>(g);\n"
      << "      const float4* t4 = reinterpret_cast<const float4*>(tile);\n"
      << "      const int64_t gb = base + toff;\n";
    for (int u = 0; u < depth; ++u)
      s << "      g4[(gb + " << hex64(deposit(uint64_t(u) << cbits)) << ") >> 1] = t4[tid + " << u * T << "u];\n";
    s << "    }\n";
  } else {
    s << "    {\n      const int64_t gb = base + toff;\n";
    for (int u = 0; u < depth; ++u)
      s << "      g[gb + " << hex64(deposit(uint64_t(u) << cbits)) << "] = A::to_store(tile[tid + " << u * T
        << "u]);\n";
    s << "    }\n";
  }
  s << "    __syncthreads();\n  }\n}\n";
  return s.str();
}

}  // namespace qs
