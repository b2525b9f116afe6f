// Kernel launches of the one-pass-per-gate path, reductions and utilities.
#include <algorithm>
#include <cmath>

#include "multi_kernels.cuh"
#include "tc_multi.cuh"
#include "pass_kernels.cuh"
#include "reduce_kernels.cuh"
#include "runtime.h"

namespace qs {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;

int grid_for(const Env& env, int64_t items, int per_thread) {
  const int64_t want = (items + int64_t(kThreads) * per_thread - 1) / (int64_t(kThreads) * per_thread);
  const int64_t cap = int64_t(env.sms) * 8;
  return int(std::max<int64_t>(1, std::min(want, cap)));
}

// Fixed-bit spec from (position, value) pairs.
Fixed make_fixed(std::vector<std::pair<int, int>> bits) {
  std::sort(bits.begin(), bits.end());
  Fixed f{};
  f.n = int(bits.size());
  f.vals = 0;
  for (int k = 0; k < f.n; ++k) {
    f.pos[k] = uint8_t(bits[k].first);
    if (bits[k].second) f.vals |= uint64_t(1) << k;
  }
  return f;
}

std::vector<std::pair<int, int>> ctrl_bits(uint64_t mask, int value) {
  std::vector<std::pair<int, int>> v;
  for (int q = 0; q < 64; ++q)
    if ((mask >> q) & 1) v.push_back({q, value});
  return v;
}

template <typename R>
Mat2<R> to_mat(const GateOp& op, double yscale = 1.0) {
  Mat2<R> g{};
  if (op.k == OpK::GEN) {
    for (int e = 0; e < 4; ++e) {
      g.re[e] = R(op.m[2 * e]);
      g.im[e] = R(op.m[2 * e + 1]);
    }
  } else if (op.k == OpK::H) {
    g.re[0] = R(1.0 / std::sqrt(2.0));
  }
  return g;
}

// The unscaled H / sqrt(X) / sqrt(Y) kernels' argument: the factor on the
// bit-1 input.
template <typename R>
Mat2<R> yscale_mat(double c) {
  Mat2<R> g{};
  g.re[0] = R(c);
  return g;
}

// Floating-point operations of one pair update (FMA counted as 2).
// GEN, H, SX, SY, X, unscaled H, SX, SY, phase-shear (two forms)
constexpr double kPairFlops[10] = {28, 8, 12, 12, 0, 4, 4, 4, 12, 12};
const char* kPairName[10] = {"gen", "h", "sx", "sy", "x", "h", "sx", "sy", "gen", "gen"};

template <typename R>
std::string kname(const char* base, const char* kind = nullptr) {
  std::string s(base);
  if (kind) s += std::string("_") + kind;
  return s + (sizeof(R) == 8 ? "_c128" : "_c64");
}

template <typename R>
constexpr double amp_bytes() { return 2.0 * sizeof(R); }

// A diagonal update on the nsel amplitudes selected by fx.  Where the
// selected amplitudes come in runs (every fixed bit at position >= 1), a
// thread takes two consecutive ones with one index computation: for
// complex64 one 16-byte access (lanes stay contiguous; measured: a 3-control
// phase flip 4755 -> 5236 GB/s), for complex128 only for phases (two 16-byte
// accesses per thread half-fill each sector per instruction, which cost
// sign flips more than the saved index work: CZ 5756 -> 5545 GB/s).
template <typename R, int K>
void launch_diag(Env& env, cvec<R>* a, int64_t nsel, const Fixed& fx, R c, R s) {
  const int low = fx.n > 0 ? fx.pos[0] : 64;  // the lowest fixed bit (positions sorted)
  const bool aligned = (reinterpret_cast<uintptr_t>(a) & 15u) == 0;
  const int V = aligned && low >= 1 && (sizeof(R) == 4 || K != DK_SIGN) ? 2 : 1;
  if (V == 2)
    k_sv_diag_v<R, K, 2, kUnroll><<<grid_for(env, nsel / 2, kUnroll), kThreads, 0, env.stream>>>(a, nsel / 2, fx,
                                                                                                   c, s);
  else
    k_sv_diag<R, K, kUnroll><<<grid_for(env, nsel, kUnroll), kThreads, 0, env.stream>>>(a, nsel, fx, c, s);
}

template <typename R, int K>
void sv_pair(Env& env, Reg& r, const GateOp& op, const Mat2<R>& g) {
  auto bits = ctrl_bits(op.cmask, 1);
  bits.push_back({op.t, 0});
  const Fixed fx = make_fixed(bits);
  const int64_t nsel = r.dim >> fx.n;
  KTimer kt(env, kname<R>("sv_pair", kPairName[K]).c_str(), double(nsel) * 4 * amp_bytes<R>(),
            double(nsel) * kPairFlops[K]);
  k_sv_pair<R, K, kUnroll><<<grid_for(env, nsel, kUnroll), kThreads, 0, env.stream>>>(
      static_cast<cvec<R>*>(r.d), nsel, int64_t(1) << op.t, fx, g);
}
template <typename R, int K>
void sv_pair(Env& env, Reg& r, const GateOp& op) {
  sv_pair<R, K>(env, r, op, to_mat<R>(op));
}

// Applies the factor Reg::qscale[t] keeps for qubit t's bit-1 half.
template <typename R>
void settle_qscale(Env& env, Reg& r, int t) {
  if (r.qscale[t] == std::complex<double>(1.0, 0.0)) return;
  const Fixed fx = make_fixed({{t, 1}});
  const int64_t nsel = r.dim >> 1;
  KTimer kt(env, kname<R>("sv_qscale").c_str(), double(nsel) * 2 * amp_bytes<R>(), double(nsel) * 6);
  launch_diag<R, DK_PHASE>(env, static_cast<cvec<R>*>(r.d), nsel, fx, R(r.qscale[t].real()),
                           R(r.qscale[t].imag()));
  r.qscale[t] = 1.0;
}

// Complex128 uncontrolled general update U on target t whose pending factor
// is w = s e^{i theta}: U' = U diag(1, e^{i theta}) (unitary) acts on
// (x, s y).  U' = g diag(1, p1) R diag(1, p2) (the fused planner's
// factorisation: g = a/|a|, p1 = (c/|c|) conj(g), p2 = -(b/|b|) conj(g),
// R = |a| [[1, -t], [t, 1]], t = |b|/|a|); p2 = cos (1 + i tan) runs as
// 1 + i tan, or, when |sin| > |cos|, p2 = sin (cot + i) as cot + i; the
// real factor f (cos or sin) times s is carried through the shear
// (x - t c y~, y~ + (t/c) x, c = f s), so the pass is 6 FMAs a pair; g |a|
// joins the register's scalar and c p1 becomes t's pending factor.  Returns
// false (nothing launched) when U' does not take that form: |a|, |b| or
// |c| near 0, t > 16, or factors that do not reproduce U' to 1e-14.
template <typename R>
bool phase_shear(Env& env, Reg& r, const GateOp& op, const std::complex<double> (&U)[4], double s) {
  using C = std::complex<double>;
  const double na = std::abs(U[0]), nb = std::abs(U[1]), nc = std::abs(U[2]);
  if (!(na > 1e-150 && nb > 1e-150 && nc > 1e-150) || nb > 16.0 * na) return false;
  const C g = U[0] / na, p1 = (U[2] / nc) * std::conj(g), p2 = -(U[1] / nb) * std::conj(g);
  const C r01 = -g * nb * p2, r10 = g * p1 * nb, r11 = g * p1 * na * p2;
  if (std::abs(r01 - U[1]) > 1e-14 || std::abs(r10 - U[2]) > 1e-14 || std::abs(r11 - U[3]) > 1e-14) return false;
  const bool by_cos = std::abs(p2.real()) >= std::abs(p2.imag());
  const double f = by_cos ? p2.real() : p2.imag();
  const double t = nb / na, c = f * s;
  Mat2<R> m{};
  m.re[0] = R(by_cos ? p2.imag() / p2.real() : p2.real() / p2.imag());
  m.re[1] = R(t * c);
  m.re[2] = R(t / c);
  if (by_cos) sv_pair<R, PK_PSP>(env, r, op, m);
  else sv_pair<R, PK_PSP2>(env, r, op, m);
  r.pend_scale *= g * na;
  r.qscale[op.t] = c * p1;
  return true;
}

// The 2x2 matrix of an uncontrolled H / sqrt(X) / sqrt(Y) / general op.
inline void op_matrix(const GateOp& op, std::complex<double> (&U)[4]) {
  using C = std::complex<double>;
  const double s = std::sqrt(0.5);
  if (op.k == OpK::GEN) {
    for (int e = 0; e < 4; ++e) U[e] = C(op.m[2 * e], op.m[2 * e + 1]);
  } else if (op.k == OpK::H) {
    U[0] = s; U[1] = s; U[2] = s; U[3] = -s;
  } else if (op.k == OpK::SX) {
    U[0] = C(0.5, 0.5); U[1] = C(0.5, -0.5); U[2] = C(0.5, -0.5); U[3] = C(0.5, 0.5);
  } else {  // sqrt(Y)
    U[0] = C(0.5, 0.5); U[1] = C(-0.5, -0.5); U[2] = C(0.5, 0.5); U[3] = C(0.5, 0.5);
  }
}

template <typename R, int K>
void dm_pair(Env& env, Reg& r, const GateOp& op) {
  const int N = r.n;
  const Fixed fx = make_fixed({{op.t, 0}, {op.t + N, 0}});
  const int64_t nsel = r.dim >> 2;
  KTimer kt(env, kname<R>("dm_quad", kPairName[K]).c_str(), double(nsel) * 8 * amp_bytes<R>(),
            double(nsel) * 4 * kPairFlops[K]);
  // (the unscaled kinds take their bit-1 factor, here 1, in g.re[0])
  const Mat2<R> g = K >= PK_HU ? yscale_mat<R>(1.0) : to_mat<R>(op);
  k_dm_gate<R, K, 2><<<grid_for(env, nsel, 2), kThreads, 0, env.stream>>>(
      static_cast<cvec<R>*>(r.d), nsel, int64_t(1) << op.t, int64_t(1) << (op.t + N), op.cmask,
      op.cmask << N, fx, g);
}

// Complex64 multi-target pass on the tensor cores (tc_multi.cuh): a
// persistent grid of 128-thread CTAs, as many per SM as can be resident.
template <int M, bool COAL>
void launch_tc(Env& env, Reg& r, const TcParams<M>& p, const Fixed& fx, int64_t nsel) {
  constexpr size_t smem = tc_smem_bytes<M>();
  // resident CTAs per SM, the least of what registers (allocated per warp
  // in units of 256), shared memory (228 KB per SM, 1 KB reserved per CTA)
  // and tensor memory (512 columns, 2^(M+1) per CTA) allow: the persistent
  // grid must be resident all at once (a function-local static: initialised
  // once, thread-safe; the serving scheduler thread may get here first)
  static const int per_sm = [] {
    QS_CUDA(cudaFuncSetAttribute(k_sv_multi_tc<M, COAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    cudaFuncAttributes fa{};
    QS_CUDA(cudaFuncGetAttributes(&fa, k_sv_multi_tc<M, COAL>));
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = 65536 / std::max(1, regs_warp * (kTcRows / 32));
    const int by_smem = int((228 * 1024) / (smem + fa.sharedSizeBytes + 1024));
    return std::max(1, std::min({by_regs, by_smem, 512 / (2 << M), 8}));
  }();
  const int64_t ntiles = (nsel + kTcRows - 1) / kTcRows;
  const int grid = int(std::min<int64_t>(ntiles, int64_t(env.sms) * per_sm));
  // algorithmic flops: 2^m complex multiply-adds (8 flops) per amplitude
  KTimer kt(env, "sv_multi_tc_c64", double(nsel) * 2 * (1 << M) * sizeof(float2),
            double(nsel) * (1 << (2 * M)) * 8);
  k_sv_multi_tc<M, COAL><<<grid, kTcRows, smem, env.stream>>>(static_cast<float2*>(r.d), nsel, fx, p,
                                                               env.d_status);
}

// The staged tensor-core pass (k_sv_multi_tcs): a persistent grid of CTAs
// (128 threads for 4 targets, 256 for 5), as many per SM as registers,
// shared memory and tensor memory (512 columns) allow.
template <int M, int MODE>
void launch_tcs(Env& env, Reg& r, const TcParams<M>& p, const Fixed& fx, int64_t nsel) {
  constexpr size_t smem = tcs_smem_bytes<M>();
  static const int per_sm = [] {
    QS_CUDA(cudaFuncSetAttribute(k_sv_multi_tcs<M, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    cudaFuncAttributes fa{};
    QS_CUDA(cudaFuncGetAttributes(&fa, k_sv_multi_tcs<M, MODE>));
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = 65536 / std::max(1, regs_warp * (kTcRows * tcs_group<M>() / 32));
    const int by_smem = int((228 * 1024) / (smem + fa.sharedSizeBytes + 1024));
    return std::max(1, std::min({by_regs, by_smem, int(512 / tcs_tmem_cols<M>()), 8}));
  }();
  const int64_t ntiles = nsel / kTcRows;
  const int grid = int(std::min<int64_t>(ntiles, int64_t(env.sms) * per_sm));
  KTimer kt(env, "sv_multi_tc_c64", double(nsel) * 2 * (1 << M) * sizeof(float2),
            double(nsel) * (1 << (2 * M)) * 8);
  k_sv_multi_tcs<M, MODE><<<grid, kTcRows * tcs_group<M>(), smem, env.stream>>>(static_cast<float2*>(r.d), nsel, fx, p,
                                                                env.d_status);
}

template <int M>
void multi_pass_tc(Env& env, Reg& r, const MultiParams<float, M>& mp, const Fixed& fx, int64_t nsel) {
  constexpr int D2 = 1 << M;
  TcParams<M> p{};
  // targets ascending: target k of the kernel is mp.t[order[k]], so bit k
  // of a kernel block index is bit order[k] of the matrix's index
  int order[M];
  for (int k = 0; k < M; ++k) order[k] = k;
  std::sort(order, order + M, [&](int x, int y) { return mp.t[x] < mp.t[y]; });
  for (int k = 0; k < M; ++k) p.t[k] = mp.t[order[k]];
  auto orig = [&](int i) {
    int o = 0;
    for (int k = 0; k < M; ++k)
      if ((i >> k) & 1) o |= 1 << order[k];
    return o;
  };
  for (int n = 0; n < D2; ++n)
    for (int l = 0; l < D2; ++l) {
      const auto& u = mp.u[orig(n) * D2 + orig(l)];
      p.u[n * D2 + l] = make_float2(u.x, u.y);
    }
  const int tmin = p.t[0];
  const bool staged = env.multi_tc_stage != 0 && nsel >= kTcRows;
  // tiles in address order (the staged kernel, or targets among the five
  // lowest qubits, where a thread's block would be runs of contiguous
  // amplitudes): the enumeration takes the 7 lowest free qubits and the
  // targets, ascending
  if ((staged || tmin < 5) && nsel >= kTcRows) {
    uint64_t fixed = 0;
    for (int k = 0; k < fx.n; ++k) fixed |= uint64_t(1) << fx.pos[k];
    std::vector<std::pair<int, int>> en;  // (qubit, role)
    for (int q = 0, j = 0; q < r.nq && j < 7; ++q)
      if (!((fixed >> q) & 1)) en.push_back({q, j++});
    for (int k = 0; k < M; ++k) en.push_back({int(p.t[k]), 0x80 | k});
    std::sort(en.begin(), en.end());
    for (size_t k = 0; k < en.size(); ++k) {
      p.pos[k] = uint8_t(en[k].first);
      p.role[k] = uint8_t(en[k].second);
    }
    if (staged) {
      p.split = p.pos[0] != 0;  // qubit 0 is a control
      // row bits 0..4 at qubits 0..4: a warp's rows are consecutive
      // amplitudes, stores straight from registers (5 targets; with 4, the
      // four CTAs an SM measured faster storing through the stage, 0.92 vs
      // 0.85 of HBM at 30 qubits); else results leave through the stage,
      // read in pairs when target 0 is at qubit 0
      bool direct = M == 5;
      for (int k = 0; k < 5; ++k) direct = direct && p.pos[k] == k && p.role[k] == k;
      const bool pair = p.pos[0] == 0 && p.role[0] == 0x80;
      if (direct) launch_tcs<M, 0>(env, r, p, fx, nsel);
      else if (pair) launch_tcs<M, 2>(env, r, p, fx, nsel);
      else launch_tcs<M, 1>(env, r, p, fx, nsel);
    } else {
      launch_tc<M, true>(env, r, p, fx, nsel);
    }
  } else {
    launch_tc<M, false>(env, r, p, fx, nsel);
  }
}

// The tiled complex64 pass (k_sv_multi_f2_tile): false (nothing launched)
// when fewer than 8 qubits are neither target nor control.
template <int M>
bool multi_pass_tile(Env& env, Reg& r, const MultiParams<float, M>& mp, uint64_t cmask) {
  uint64_t tmask = 0;
  for (int k = 0; k < M; ++k) tmask |= uint64_t(1) << mp.t[k];
  std::vector<int> fq;  // the 8 lowest free qubits
  for (int q = 0; q < r.nq && int(fq.size()) < 8; ++q)
    if (!((tmask >> q) & 1) && !((cmask >> q) & 1)) fq.push_back(q);
  if (fq.size() < 8) return false;
  std::vector<int> L;  // local qubits, ascending
  for (int q = 0; q < r.nq; ++q)
    if (((tmask >> q) & 1) || std::find(fq.begin(), fq.end(), q) != fq.end()) L.push_back(q);
  auto local_of = [&](int q) { return int(std::find(L.begin(), L.end(), q) - L.begin()); };
  MultiTileParams<M> p{};
  for (int k = 0; k < M + 8; ++k) p.lpos[k] = uint8_t(L[size_t(k)]);
  for (int j = 0; j < 8; ++j) p.fpos[j] = uint8_t(local_of(fq[size_t(j)]));
  // bank bits: a half-warp's 16 blocks differ in block-index bits 0..3; give
  // each of their local bits at position >= 4 a bank bit the others lack
  uint32_t used = 0;
  for (int j = 0; j < 4; ++j)
    if (p.fpos[j] < 4) used |= 1u << p.fpos[j];
  for (int j = 0; j < 4; ++j)
    if (p.fpos[j] >= 4) {
      int e = 0;
      while ((used >> e) & 1u) ++e;
      p.swz[p.fpos[j]] = uint8_t(1u << e);
      used |= 1u << e;
    }
  auto slot = [&](uint32_t x) {
    uint32_t s = x;
    for (int k = 4; k < M + 8; ++k)
      if ((x >> k) & 1u) s ^= p.swz[k];
    return uint16_t(s);
  };
  for (int i = 0; i < (1 << M); ++i) {
    int64_t g = 0;
    for (int k = 0; k < M; ++k)
      if ((i >> k) & 1) g += int64_t(1) << L[size_t(8 + k)];
    p.goff_hi[i] = g;
    p.sm_hi[i] = slot(uint32_t(i) << 8);
    uint32_t lam = 0;
    for (int k = 0; k < M; ++k)
      if ((i >> k) & 1) lam |= 1u << local_of(mp.t[k]);
    p.sm_l[i] = slot(lam);
  }
  for (int e = 0; e < (1 << (2 * M)); ++e)
    p.u[e] = make_float4(mp.u[e].x, mp.u[e].x, mp.u[e].y, mp.u[e].y);
  std::vector<std::pair<int, int>> bits = ctrl_bits(cmask, 1);
  for (int q : L) bits.push_back({q, 0});
  const Fixed fx = make_fixed(bits);
  const int64_t ntiles = r.dim >> fx.n;
  // one wave of resident CTAs (each prefetches its next tile)
  static const int per_sm = [] {
    int nb = 0;
    QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sv_multi_f2_tile<M>, 256, 0));
    return std::max(1, nb);
  }();
  const int grid = int(std::min<int64_t>(ntiles, int64_t(env.sms) * per_sm));
  KTimer kt(env, "sv_multi_c64", double(ntiles) * 256 * 2 * (1 << M) * sizeof(float2),
            double(ntiles) * 256 * (1 << (2 * M)) * 8);
  k_sv_multi_f2_tile<M><<<grid, 256, 0, env.stream>>>(static_cast<float2*>(r.d), ntiles, fx, p);
  return true;
}

// One multi-target pass over the vector: targets t (shifted by `shift`),
// controls cmask, matrix (conjugated when conj).
template <typename R, int M>
void multi_pass(Env& env, Reg& r, const GateOp& op, int shift, uint64_t cmask, bool conj) {
  MultiParams<R, M> p{};
  std::vector<std::pair<int, int>> bits = ctrl_bits(cmask, 1);
  for (int k = 0; k < M; ++k) {
    p.t[k] = uint8_t(op.tg[k] + shift);
    bits.push_back({op.tg[k] + shift, 0});
  }
  const std::vector<double>& u = *op.big;
  for (int e = 0; e < (1 << (2 * M)); ++e) {
    p.u[e].x = R(u[2 * e]);
    p.u[e].y = R(conj ? -u[2 * e + 1] : u[2 * e + 1]);
  }
  const Fixed fx = make_fixed(bits);
  const int64_t nsel = r.dim >> fx.n;
  if constexpr (std::is_same<R, float>::value) {
    // by shape: 5 targets on the tensor cores, and 4 where the staged
    // tensor-core kernel runs (at least 7 free qubits); else up to 4 on the
    // CUDA cores (paired FMAs), at 3-4 through shared-memory tiles when a
    // target is among the five lowest qubits (a thread's block would be
    // short contiguous runs)
    int tmin = 64;
    for (int k = 0; k < M; ++k) tmin = std::min(tmin, int(p.t[k]));
    if constexpr (M >= 4) {
      const bool staged = env.multi_tc_stage != 0 && nsel >= kTcRows;
      if (env.multi_tc == 2 || (env.multi_tc == 1 && (M == 5 || staged))) {
        multi_pass_tc<M>(env, r, p, fx, nsel);
        return;
      }
    }
    if constexpr (M >= 3 && M <= 4) {  // (at 2 targets the per-block loads do as well)
      if (tmin < 5 && multi_pass_tile<M>(env, r, p, cmask)) return;
    }
  }
  KTimer kt(env, kname<R>("sv_multi").c_str(), double(nsel) * 2 * (1 << M) * amp_bytes<R>(),
            double(nsel) * (1 << (2 * M)) * 8);
  // complex64 on up to 4 targets with paired FP32 FMAs; at 5 targets the
  // duplicated matrix (16 KB of parameters) is fetched into registers entry by
  // entry, slower than the scalar kernel whose FMAs read it as operands
  if constexpr (std::is_same<R, double>::value) {
    if (env.arith == 1) {  // double-float on the FP32 pipes
      MultiParamsDF<M> q{};
      for (int k = 0; k < 8; ++k) q.t[k] = p.t[k];
      for (int e = 0; e < (1 << (2 * M)); ++e) {
        const double re = u[2 * e], im = conj ? -u[2 * e + 1] : u[2 * e + 1];
        const float rh = float(re), ih = float(im);
        q.u[e] = make_float4(rh, float(re - double(rh)), ih, float(im - double(ih)));
      }
      k_sv_multi_df<M><<<grid_for(env, nsel, 1), kThreads, 0, env.stream>>>(static_cast<double2*>(r.d), nsel,
                                                                             fx, q);
      return;
    }
  }
  if constexpr (std::is_same<R, float>::value && M <= 4) {
    MultiParamsF2<M> q{};
    for (int k = 0; k < 8; ++k) q.t[k] = p.t[k];
    for (int e = 0; e < (1 << (2 * M)); ++e) q.u[e] = make_float4(p.u[e].x, p.u[e].x, p.u[e].y, p.u[e].y);
    k_sv_multi_f2<M><<<grid_for(env, nsel, 1), kThreads, 0, env.stream>>>(static_cast<float2*>(r.d), nsel, fx, q);
    return;
  }
  k_sv_multi<R, M><<<grid_for(env, nsel, 1), kThreads, 0, env.stream>>>(static_cast<cvec<R>*>(r.d), nsel,
                                                                        fx, p);
}

template <typename R, int M>
void multi_op(Env& env, Reg& r, const GateOp& op) {
  for (int k = 0; k < M; ++k) settle_qscale<R>(env, r, op.tg[k]);
  multi_pass<R, M>(env, r, op, 0, op.cmask, false);
  if (r.density) multi_pass<R, M>(env, r, op, r.n, op.cmask << r.n, true);
}

template <typename R>
void launch_typed(Env& env, Reg& r, const GateOp& op) {
  cvec<R>* a = static_cast<cvec<R>*>(r.d);
  if (op.k == OpK::MULTI) {
    if (op.nt == 1) {  // a 2x2 update: the single-target path (pair kernels, phase-shear)
      GateOp g = op;
      g.k = OpK::GEN;
      g.t = op.tg[0];
      g.nt = 0;
      const std::vector<double>& u = *op.big;
      for (int e = 0; e < 8; ++e) g.m[e] = u[size_t(e)];
      g.big.reset();
      launch_typed<R>(env, r, g);
      return;
    }
    switch (op.nt) {
      case 1: multi_op<R, 1>(env, r, op); return;
      case 2: multi_op<R, 2>(env, r, op); return;
      case 3: multi_op<R, 3>(env, r, op); return;
      case 4: multi_op<R, 4>(env, r, op); return;
      case 5: multi_op<R, 5>(env, r, op); return;
      default: fail(QS_E_ARG, "1..5 targets supported");
    }
  }
  if (!r.density) {
    // a pair update on target t needs t's deferred bit-1 factor applied first,
    // unless it takes it as its bit-1 input factor (uncontrolled H / sqrt(X) /
    // sqrt(Y) below)
    // (sign flips have no target: op.t = -1)
    const bool real_pending = op.t < 0 || r.qscale[op.t].imag() == 0.0;
    const bool hsxsy = op.k == OpK::H || op.k == OpK::SX || op.k == OpK::SY;
    // complex128, uncontrolled general update (or H / sqrt(X) / sqrt(Y) meeting a
    // complex pending factor): phase-shear with the pending factor folded in
    const bool ps_path = sizeof(R) == 8 && op.cmask == 0 && (op.k == OpK::GEN || (hsxsy && !real_pending));
    // uncontrolled H / sqrt(X) / sqrt(Y) with a real pending factor: its bit-1 input factor
    const bool yscale_path = op.cmask == 0 && hsxsy && real_pending;
    if ((op.k == OpK::GEN || op.k == OpK::X || hsxsy) && !ps_path && !yscale_path) settle_qscale<R>(env, r, op.t);
    if (ps_path) {
      std::complex<double> U[4];
      op_matrix(op, U);
      const std::complex<double> w = r.qscale[op.t];
      const double sw = std::abs(w);
      std::complex<double> Up[4] = {U[0], U[1] * (w / sw), U[2], U[3] * (w / sw)};
      if (!phase_shear<R>(env, r, op, Up, sw)) {
        U[1] *= w;
        U[3] *= w;
        GateOp g = op;  // the plain general update of U diag(1, w)
        g.k = OpK::GEN;
        for (int e = 0; e < 4; ++e) {
          g.m[2 * e] = U[e].real();
          g.m[2 * e + 1] = U[e].imag();
        }
        sv_pair<R, PK_GEN>(env, r, g);
        r.qscale[op.t] = 1.0;
      }
      if (std::abs(r.qscale[op.t]) < 1e-100) settle_qscale<R>(env, r, op.t);
      return;
    }
    switch (op.k) {
      case OpK::GEN: sv_pair<R, PK_GEN>(env, r, op); return;
      // uncontrolled H / sqrt(X) / sqrt(Y): unscaled, the register keeps the
      // scalar factor; the bit-1 input takes the qubit's deferred factor
      case OpK::H:
      case OpK::SX:
      case OpK::SY: {
        if (op.cmask) {
          if (op.k == OpK::H) sv_pair<R, PK_H>(env, r, op);
          else if (op.k == OpK::SX) sv_pair<R, PK_SX>(env, r, op);
          else sv_pair<R, PK_SY>(env, r, op);
          return;
        }
        const Mat2<R> g = yscale_mat<R>(r.qscale[op.t].real());
        r.qscale[op.t] = 1.0;
        if (op.k == OpK::H) {
          sv_pair<R, PK_HU>(env, r, op, g);
          r.pend_scale *= std::sqrt(0.5);
        } else {
          if (op.k == OpK::SX) sv_pair<R, PK_SXU>(env, r, op, g);
          else sv_pair<R, PK_SYU>(env, r, op, g);
          r.pend_scale *= std::complex<double>(0.5, 0.5);
        }
        return;
      }
      case OpK::X: sv_pair<R, PK_X>(env, r, op); return;
      case OpK::PHASE: {
        auto bits = ctrl_bits(op.cmask, 1);
        bits.push_back({op.t, 1});
        const Fixed fx = make_fixed(bits);
        const int64_t nsel = r.dim >> fx.n;
        // complex128, uncontrolled: (1 + i tan phi) on the bit-1 half (2 FP64
        // FMAs instead of 4 operations, the FP64 pipe being the bound); cos phi
        // joins the qubit's deferred factor (a diagonal factor commutes with
        // every op that does not target the qubit)
        if (sizeof(R) == 8 && op.cmask == 0 && std::abs(op.m[0]) >= 0.5) {
          KTimer kt(env, kname<R>("sv_phase").c_str(), double(nsel) * 2 * amp_bytes<R>(), double(nsel) * 4);
          launch_diag<R, DK_PHASEU>(env, a, nsel, fx, R(1), R(op.m[1] / op.m[0]));
          r.qscale[op.t] *= op.m[0];
          if (std::abs(r.qscale[op.t]) < 1e-100) settle_qscale<R>(env, r, op.t);
          return;
        }
        KTimer kt(env, kname<R>("sv_phase").c_str(), double(nsel) * 2 * amp_bytes<R>(), double(nsel) * 6);
        launch_diag<R, DK_PHASE>(env, a, nsel, fx, R(op.m[0]), R(op.m[1]));
        return;
      }
      case OpK::SIGN: {
        const Fixed fx = make_fixed(ctrl_bits(op.cmask, 1));
        const int64_t nsel = r.dim >> fx.n;
        KTimer kt(env, kname<R>("sv_sign").c_str(), double(nsel) * 2 * amp_bytes<R>(), 0);
        launch_diag<R, DK_SIGN>(env, a, nsel, fx, R(0), R(0));
        return;
      }
      default: fail(QS_E_NOT_DENSITY, "channel on a state vector");
    }
  }
  const int N = r.n;
  switch (op.k) {
    case OpK::GEN: dm_pair<R, PK_GEN>(env, r, op); return;
    // uncontrolled: unscaled row and column updates, factor |f|^2 = 1/2 kept
    case OpK::H:
    case OpK::SX:
    case OpK::SY:
      if (op.cmask) {
        if (op.k == OpK::H) dm_pair<R, PK_H>(env, r, op);
        else if (op.k == OpK::SX) dm_pair<R, PK_SX>(env, r, op);
        else dm_pair<R, PK_SY>(env, r, op);
        return;
      }
      if (op.k == OpK::H) dm_pair<R, PK_HU>(env, r, op);
      else if (op.k == OpK::SX) dm_pair<R, PK_SXU>(env, r, op);
      else dm_pair<R, PK_SYU>(env, r, op);
      r.pend_scale *= 0.5;
      return;
    case OpK::X: dm_pair<R, PK_X>(env, r, op); return;
    case OpK::PHASE: {
      KTimer kt(env, kname<R>("dm_phase").c_str(), double(r.dim) * amp_bytes<R>(), double(r.dim) * 3);
      k_dm_diag<R, DD_PHASE><<<grid_for(env, r.dim, 1), kThreads, 0, env.stream>>>(
          a, r.dim, N, op.cmask, op.t, R(op.m[0]), R(op.m[1]));
      return;
    }
    case OpK::SIGN: {
      const double f = std::ldexp(1.0, -__builtin_popcountll(op.cmask));
      KTimer kt(env, kname<R>("dm_sign").c_str(), double(r.dim) * 4 * f * (1 - f) * amp_bytes<R>(), 0);
      k_dm_diag<R, DD_SIGN><<<grid_for(env, r.dim, 1), kThreads, 0, env.stream>>>(
          a, r.dim, N, op.cmask, 0, R(0), R(0));
      return;
    }
    case OpK::DEPHASE: {
      KTimer kt(env, kname<R>("dm_dephase").c_str(), double(r.dim) * amp_bytes<R>(), double(r.dim));
      k_dm_diag<R, DD_DEPHASE><<<grid_for(env, r.dim, 1), kThreads, 0, env.stream>>>(
          a, r.dim, N, 0, op.t, R(1.0 - 2.0 * op.m[0]), R(0));
      return;
    }
    case OpK::DEPOL: {
      const double p = op.m[0];
      const Fixed fx = make_fixed({{op.t, 0}, {op.t + N, 0}});
      const int64_t nsel = r.dim >> 2;
      KTimer kt(env, kname<R>("dm_depol").c_str(), double(nsel) * 8 * amp_bytes<R>(), double(nsel) * 16);
      k_dm_depol<R, 2><<<grid_for(env, nsel, 2), kThreads, 0, env.stream>>>(
          a, nsel, int64_t(1) << op.t, int64_t(1) << (op.t + N), fx, R(1.0 - 2.0 * p / 3.0),
          R(2.0 * p / 3.0), R(1.0 - 4.0 * p / 3.0));
      return;
    }
  }
}

void check_launch() { QS_CUDA(cudaGetLastError()); }

template <typename R>
void sumsq(Env& env, const Reg& r, const Fixed& fx, int64_t nsel, double* out) {
  // one block up to 16 amplitudes a thread (registers of up to 2^13
  // amplitudes): its partial is the result, so the second stage (which would
  // add zeros to it) is skipped, saving a launch
  const int blocks = nsel <= int64_t(kRedThreads) * 16
                         ? 1
                         : int(std::min<int64_t>(kRedMaxBlocks, (nsel + kRedThreads * 4 - 1) / (kRedThreads * 4)));
  KTimer kt(env, kname<R>("reduce_sumsq").c_str(), double(nsel) * amp_bytes<R>(), double(nsel) * 4,
            blocks == 1 ? 1 : 2);
  k_sumsq<R, 4><<<blocks, kRedThreads, 0, env.stream>>>(static_cast<const cvec<R>*>(r.d), nsel, fx,
                                                        blocks == 1 ? out : env.d_partial);
  if (blocks > 1) k_sum_partials<<<1, 1024, 0, env.stream>>>(env.d_partial, blocks, out);
}

template <typename R>
void sumdiag(Env& env, const Reg& r, int q, int o, double* out) {
  const int64_t d = int64_t(1) << r.n;
  const int blocks = int(std::max<int64_t>(
      1, std::min<int64_t>(kRedMaxBlocks, (d + kRedThreads - 1) / kRedThreads)));
  KTimer kt(env, kname<R>("reduce_diag").c_str(), double(d) * amp_bytes<R>(), double(d), blocks == 1 ? 1 : 2);
  k_sumdiag<R><<<blocks, kRedThreads, 0, env.stream>>>(static_cast<const cvec<R>*>(r.d), r.n, q, o,
                                                       blocks == 1 ? out : env.d_partial);
  if (blocks > 1) k_sum_partials<<<1, 1024, 0, env.stream>>>(env.d_partial, blocks, out);
}

double fetch_result(Env& env) {
  check_launch();
  QS_CUDA(cudaMemcpyAsync(env.h_result, env.d_result, sizeof(double), cudaMemcpyDeviceToHost,
                          env.stream));
  QS_CUDA(cudaMemcpyAsync(env.h_status, env.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, env.stream));
  QS_CUDA(cudaStreamSynchronize(env.stream));
  check_status(env);
  return env.h_result[0];
}

}  // namespace

void launch_wait_probe(Env& env, int timeout_us) {
  k_wait_probe<<<1, 32, 0, env.stream>>>(env.d_status, uint64_t(timeout_us) * 1000u);
  check_launch();
}

void settle_qscales(Reg& r) {
  for (int t = 0; t < r.nq; ++t) {
    if (r.qscale[t] == 1.0) continue;
    if (r.prec == QS_C128) settle_qscale<double>(*r.env, r, t);
    else settle_qscale<float>(*r.env, r, t);
  }
}

void check_status(Env& env) {
  const unsigned s = *env.h_status;
  if (s == 0) return;
  *env.h_status = 0;
  QS_CUDA(cudaMemsetAsync(env.d_status, 0, sizeof(unsigned), env.stream));
  fail(QS_E_TIMEOUT, std::string("a bounded device wait ran out (") +
                         ((s & 1u)   ? "tensor-core multi-target pass"
                          : (s & 2u) ? "bulk tile copy of a fused pass"
                                     : "persistent batch: a register's previous pass") +
                         "); amplitudes are unreliable");
}

// Unscaled passes grow the stored amplitudes by 1/|pend_scale|: settle the
// factor before that growth nears the storage format's range.  Unitary
// updates keep the stored vector's norm at 1/|pend_scale|, so no stored
// amplitude exceeds it: 1e18 for complex64 (float range 3.4e38), 1e100 for
// complex128; precision is relative and does not depend on the scale.
static void bound_pending(Env& env, Reg& r) {
  if (std::abs(r.pend_scale) >= (r.prec == QS_C64 ? 1e-18 : 1e-100)) return;
  launch_scale(env, r, r.pend_scale);
  r.pend_scale = 1.0;
}

static void launch_op_impl(Env& env, Reg& r, const GateOp& op);

void launch_op(Env& env, Reg& r, const GateOp& op) {
  launch_op_impl(env, r, op);
  bound_pending(env, r);
}

static void launch_op_impl(Env& env, Reg& r, const GateOp& op) {
  if (r.prec == QS_C128) launch_typed<double>(env, r, op);
  else launch_typed<float>(env, r, op);
  check_launch();
}

void queue_total(Env& env, Reg& r, double* out) {
  flush(r);
  if (r.density) {
    if (r.prec == QS_C128) sumdiag<double>(env, r, -1, 0, out);
    else sumdiag<float>(env, r, -1, 0, out);
  } else {
    const Fixed fx = make_fixed({});
    if (r.prec == QS_C128) sumsq<double>(env, r, fx, r.dim, out);
    else sumsq<float>(env, r, fx, r.dim, out);
  }
  check_launch();
}

void queue_outcome(Env& env, Reg& r, int q, int o, double* out) {
  flush(r);
  if (r.density) {
    if (r.prec == QS_C128) sumdiag<double>(env, r, q, o, out);
    else sumdiag<float>(env, r, q, o, out);
  } else {
    const Fixed fx = make_fixed({{q, o}});
    if (r.prec == QS_C128) sumsq<double>(env, r, fx, r.dim >> 1, out);
    else sumsq<float>(env, r, fx, r.dim >> 1, out);
  }
  check_launch();
}

namespace {
template <typename RA, typename RB>
void inner(Env& env, const Reg& a, const Reg& b, double* out) {
  const int blocks = int(std::max<int64_t>(
      1, std::min<int64_t>(kRedMaxBlocks, (a.dim + kRedThreads * 4 - 1) / (kRedThreads * 4))));
  KTimer kt(env, "reduce_inner", double(a.dim) * (amp_bytes<RA>() + amp_bytes<RB>()), double(a.dim) * 8, 3);
  k_inner<RA, RB, 4><<<blocks, kRedThreads, 0, env.stream>>>(static_cast<const cvec<RA>*>(a.d),
                                                            static_cast<const cvec<RB>*>(b.d), a.dim,
                                                            env.d_partial);
  k_sum_partials<<<1, 1024, 0, env.stream>>>(env.d_partial, blocks, out);
  k_sum_partials<<<1, 1024, 0, env.stream>>>(env.d_partial + blocks, blocks, out + 1);
}
}  // namespace

std::complex<double> reduce_inner(Env& env, Reg& a, Reg& b) {
  flush(a);
  flush(b);
  // both registers' pending work must be done before the reduction reads
  // them: b's env may queue on another stream
  if (b.env != &env) QS_CUDA(cudaStreamSynchronize(b.env->stream));
  if (a.prec == QS_C128 && b.prec == QS_C128) inner<double, double>(env, a, b, env.d_result);
  else if (a.prec == QS_C128) inner<double, float>(env, a, b, env.d_result);
  else if (b.prec == QS_C128) inner<float, double>(env, a, b, env.d_result);
  else inner<float, float>(env, a, b, env.d_result);
  check_launch();
  QS_CUDA(cudaMemcpyAsync(env.h_result, env.d_result, 2 * sizeof(double), cudaMemcpyDeviceToHost, env.stream));
  QS_CUDA(cudaMemcpyAsync(env.h_status, env.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, env.stream));
  QS_CUDA(cudaStreamSynchronize(env.stream));
  check_status(env);
  return {env.h_result[0], env.h_result[1]};
}

double reduce_total(Env& env, Reg& r) {
  queue_total(env, r, env.d_result);
  return fetch_result(env);
}

double reduce_outcome(Env& env, Reg& r, int q, int o) {
  queue_outcome(env, r, q, o, env.d_result);
  return fetch_result(env);
}

double reduce_purity(Env& env, Reg& r) {
  flush(r);
  const Fixed fx = make_fixed({});
  if (r.prec == QS_C128) sumsq<double>(env, r, fx, r.dim, env.d_result);
  else sumsq<float>(env, r, fx, r.dim, env.d_result);
  return fetch_result(env);
}

void launch_collapse(Env& env, Reg& r, int q, int o, double scale) {
  const int g = grid_for(env, r.dim, 1);
  const double keep = r.density ? 0.25 : 0.5;
  KTimer kt(env, r.prec == QS_C128 ? "collapse_c128" : "collapse_c64",
            double(r.dim) * (1 + keep) * (r.prec == QS_C128 ? 16 : 8), double(r.dim) * keep * 2);
  if (r.density) {
    if (r.prec == QS_C128)
      k_collapse_dm<double><<<g, kThreads, 0, env.stream>>>(static_cast<double2*>(r.d), r.dim, r.n, q, o, scale);
    else
      k_collapse_dm<float><<<g, kThreads, 0, env.stream>>>(static_cast<float2*>(r.d), r.dim, r.n, q, o, scale);
  } else {
    if (r.prec == QS_C128)
      k_collapse_sv<double><<<g, kThreads, 0, env.stream>>>(static_cast<double2*>(r.d), r.dim, q, o, scale);
    else
      k_collapse_sv<float><<<g, kThreads, 0, env.stream>>>(static_cast<float2*>(r.d), r.dim, q, o, scale);
  }
  check_launch();
}

void launch_fill(Env& env, Reg& r, double re, double im) {
  const int g = grid_for(env, r.dim, 1);
  KTimer kt(env, r.prec == QS_C128 ? "fill_c128" : "fill_c64", double(r.dim) * (r.prec == QS_C128 ? 16 : 8), 0);
  if (r.prec == QS_C128)
    k_fill<double><<<g, kThreads, 0, env.stream>>>(static_cast<double2*>(r.d), r.dim, re, im);
  else
    k_fill<float><<<g, kThreads, 0, env.stream>>>(static_cast<float2*>(r.d), r.dim, float(re), float(im));
  check_launch();
}

void launch_scale(Env& env, Reg& r, std::complex<double> f) {
  const int g = grid_for(env, r.dim, 1);
  KTimer kt(env, r.prec == QS_C128 ? "scale_c128" : "scale_c64",
            2.0 * double(r.dim) * (r.prec == QS_C128 ? 16 : 8), 6.0 * double(r.dim));
  if (r.prec == QS_C128)
    k_scale<double><<<g, kThreads, 0, env.stream>>>(static_cast<double2*>(r.d), r.dim, f.real(), f.imag());
  else
    k_scale<float><<<g, kThreads, 0, env.stream>>>(static_cast<float2*>(r.d), r.dim, float(f.real()),
                                                   float(f.imag()));
  check_launch();
}

__global__ void k_f2d(const float2* __restrict__ s, double2* __restrict__ d, int64_t count) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < count; n += nthr) {
    const float2 v = s[n];
    d[n] = make_double2(double(v.x), double(v.y));
  }
}

__global__ void k_d2f(const double2* __restrict__ s, float2* __restrict__ d, int64_t count) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < count; n += nthr) {
    const double2 v = s[n];
    d[n] = make_float2(float(v.x), float(v.y));
  }
}

void launch_convert(Env& env, const void* src, void* dst, int64_t count, bool to_double) {
  const int g = grid_for(env, count, 1);
  KTimer kt(env, "convert", double(count) * 24, 0);
  if (to_double)
    k_f2d<<<g, kThreads, 0, env.stream>>>(static_cast<const float2*>(src), static_cast<double2*>(dst), count);
  else
    k_d2f<<<g, kThreads, 0, env.stream>>>(static_cast<const double2*>(src), static_cast<float2*>(dst), count);
  check_launch();
}

}  // namespace qs
