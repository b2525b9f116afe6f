/*
 * qsim.h -- C ABI of the B300 exact quantum-circuit simulator.
 *
 * The library holds n-qubit state vectors (2^n complex amplitudes) and
 * N-qubit density matrices (stored as 2N-qubit vectors of 2^(2N)
 * amplitudes) in GPU memory and updates them with hand-written sm_103a
 * CUDA kernels.  Call names and call order follow the paper (QuEST,
 * arXiv 1802.08032): an environment, registers created in it, gates applied
 * one call each, and a sync that waits for the work (Sec. III,
 * "Configuration and timing").
 *
 * Conventions common to every call
 *  - Qubit q is bit q of the amplitude index (Sec. II.B.1, Eq. 1).
 *  - Amplitudes are interleaved complex numbers (re, im), contiguous:
 *    QS_C128 = two IEEE doubles (16 B), QS_C64 = two IEEE floats (8 B).
 *  - A density matrix rho of N qubits lives at index j + 2^N k for the
 *    entry rho[j][k] (row j in the low N bits, column k in the high N bits);
 *    a gate G on qubit q is enacted as G on bit q then conj(G) on bit q+N
 *    (Sec. II.B.1, Eq. 2).
 *  - Every call returns QS_OK (0) or a negative QS_E_* code; the message of
 *    the last failure on the calling thread is qsLastError().  Arguments are
 *    validated before any work is queued, so a call that fails leaves the
 *    register unchanged.
 *  - Gate and channel calls are asynchronous: they are queued on the
 *    environment's CUDA stream in call order.  Calls that return a value to
 *    the host (calcTotalProb, calcProbOfOutcome, collapseToOutcome,
 *    calcPurity, copyStateToHost) wait for the queued work.  syncQuESTEnv
 *    waits for everything and reports asynchronous device errors.
 *  - Matrices and control arrays are copied at call time; host buffers
 *    passed in stay owned by the caller.  Register memory is owned by the
 *    library (allocated through the allocator hook when one is set).
 *  - Handles are plain integers; a destroyed or unknown handle gives
 *    QS_E_HANDLE.  Calls on one environment must not race from several host
 *    threads.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } Complex;
/* Row-major 2x2 complex matrix: m[row][column]. */
typedef struct { Complex m[2][2]; } ComplexMatrix2;
/* Row-major 4x4 complex matrix (two-qubit gates). */
typedef struct { Complex m[4][4]; } ComplexMatrix4;
typedef struct { int64_t id; } QuESTEnv;
typedef struct { int64_t id; } Qureg;

/* Amplitude precision of a register. */
enum { QS_C64 = 64, QS_C128 = 128 };

/* Status codes. */
enum {
    QS_OK = 0,
    QS_E_QUBIT = -1,        /* qubit index out of range                        */
    QS_E_DUP = -2,          /* repeated qubit among targets and controls       */
    QS_E_UNITARY = -3,      /* matrix not unitary within 1e-10                 */
    QS_E_PROB = -4,         /* probability / outcome argument out of range     */
    QS_E_NOT_DENSITY = -5,  /* channel or purity on a state vector            */
    QS_E_ZERO_PROB = -6,    /* collapse onto an outcome of probability ~0      */
    QS_E_NOMEM = -7,        /* allocation failed or memory budget exceeded     */
    QS_E_HANDLE = -8,       /* unknown or destroyed handle                     */
    QS_E_CUDA = -9,         /* CUDA runtime error (message in qsLastError)     */
    QS_E_TIMEOUT = -10,     /* a bounded device or host wait ran out           */
    QS_E_ARG = -11,         /* other invalid argument (null pointer, range)    */
    QS_E_BUSY = -12         /* refused or shed by a server's admission policy  */
};

/* Message of the last failed call on this thread ("" if none). */
const char *qsLastError(void);
/* qsJitShutdown: waits for the background compiles of generated pass
 * kernels that are in flight, drops the queued ones and stops the compile
 * threads (compiled kernels stay cached; the threads start again when
 * needed).  Destroying the last environment does this; a program that exits
 * with environments alive calls it first (the Python binding does so at
 * interpreter exit): a compile still running while the process tears down
 * can crash it. */
int qsJitShutdown(void);

/* ------------------------------------------------------------ environment */
/* createQuESTEnv: binds the current CUDA device, creates a stream owned by
 * the environment (Sec. III: createQuESTEnv). */
int createQuESTEnv(QuESTEnv *out);
/* destroyQuESTEnv: waits for queued work, frees every register of the env. */
int destroyQuESTEnv(QuESTEnv env);
/* syncQuESTEnv: flushes every register's queued gates and waits for the
 * stream (Sec. III: syncQuESTEnv closes the timed region).  Returns
 * QS_E_CUDA on an asynchronous device error, QS_E_TIMEOUT when a kernel
 * reported a bounded device wait that ran out since the last check (the
 * tensor-core pass of multi-target gates waits on its MMAs; the affected
 * amplitudes are unreliable).  Reductions report the same at their next
 * result. */
int syncQuESTEnv(QuESTEnv env);
/* qsDiagBoundedWait: diagnostic of the device failure path.  Launches, on
 * the env's stream, one CTA that runs the bounded wait the tensor-core
 * multi-target pass uses (there: 1 s), on an mbarrier nothing arrives on,
 * for timeoutUs (1..10^6) microseconds of the GPU's global timer; it then
 * sets the device status word, so the next syncQuESTEnv (or reduction)
 * returns QS_E_TIMEOUT and clears it.  No fault, no unbounded wait; the
 * context stays usable.  QS_E_ARG for a timeoutUs outside the range. */
int qsDiagBoundedWait(QuESTEnv env, int timeoutUs);
/* setEnvOption: runtime options (values are integers).
 *   "fusion"        0 = one kernel pass per gate, 1 = queue gates and apply
 *                   them in shared-memory tiles at flush time (default 1).
 *                   The flush planner rewrites the queued gates exactly
 *                   (consecutive phases merge, gates on qubits still in |0>
 *                   since the register was zeroed become copies or vanish,
 *                   general 2x2 gates run as phase-rotation-phase, scalar
 *                   factors are applied once per flush; on a density matrix
 *                   the channels' off-diagonal factors are deferred per
 *                   qubit and applied with the next gate on it, and a
 *                   gate's row and column phases act on the off-diagonal
 *                   entries only): results equal applying the gates one by
 *                   one up to rounding.
 *   "tile_qubits"   k of a fused tile, 0 = automatic
 *   "fused_cluster" registers that fit one fused tile (complex128 up to 12
 *                   stored qubits, complex64 up to 13; plain arithmetic)
 *                   run it on a thread-block cluster of up to this many CTAs
 *                   (2, 4 or 8; default 8): each CTA holds a slice of the
 *                   tile in shared memory and stages reach the others'
 *                   slices through distributed shared memory, with fewer
 *                   register amplitudes a thread so that every CTA runs 4
 *                   warps.  0 or 1 = one CTA (tiles one qubit smaller on
 *                   registers of at most 18 qubits).  Amplitudes equal the
 *                   one-CTA plan's up to rounding (commuting operations may
 *                   be grouped into stages in another order); each plan is
 *                   deterministic.  Applies when "tile_qubits" is 0 or at least
 *                   the register's qubits.  Batches never use clusters.
 *   "batch_persistent" batches created (or re-tuned) from now on: 0 = one
 *                   launch per wave, captured in the batch's graph; 1 = one
 *                   persistent launch over every wave (default):
 *                   CTAs claim runs of work items from a global ticket in
 *                   wave order and, before a register's next pass, wait
 *                   until every tile of its previous pass is done (waits
 *                   bounded by 1 s of the GPU's global timer; a wait that
 *                   runs out stops the launch and the next getBatchNorms,
 *                   syncQuESTEnv or reduction returns QS_E_TIMEOUT).  The
 *                   amplitudes are the same bit for bit.
 *   "batch_diag_stall" diagnostic of that bounded wait: batches built while
 *                   it is 1 (persistent form) wait for one tile more than
 *                   each previous pass has, with a 2 ms bound instead of
 *                   1 s, so the first such wait runs out; the next
 *                   getBatchNorms returns QS_E_TIMEOUT and the context stays
 *                   usable.  Default 0.
 *   "tile_low_qubits" lowest qubits every fused tile holds: HBM chunks of
 *                   2^L contiguous amplitudes (0 = automatic: 4 for
 *                   complex64, 3 for complex128; else 2..6).  Fewer leave
 *                   more tile qubits to a pass, with shorter chunks
 *                   (measured slower below the default).
 *   "max_fused_ops" cap on operations per fused pass (0 = automatic)
 *   "budget_bytes"  cap on the register memory of this env (0 = none)
 *   "arith"         complex128 arithmetic of fused passes and multi-target
 *                   passes: 0 = IEEE FP64 (default), 1 = double-float, an
 *                   OUT-OF-SPEC precision form, not complex128 arithmetic:
 *                   each real is a float pair hi + lo on the FP32 pipes (a
 *                   48-bit significand: a few units of 2^-48 of error per
 *                   update instead of 2^-53; a multi-target pass on m
 *                   targets up to 2^m units of 2^-48 of the norm).  Storage
 *                   stays complex128; amplitudes meet the 1e-12 bar and the
 *                   FP64-reduced probabilities of the 30-qubit 1259-gate
 *                   circuit stay within 6e-14 of an FP64 oracle, but every
 *                   pass boundary rounds the float pairs to doubles, so
 *                   longer circuits with more passes drift further than IEEE
 *                   FP64.  Single-gate passes, reductions and measurement
 *                   always use FP64.
 *   "profile"       1 = time every kernel launch with CUDA events (see
 *                   getKernelStats), 0 = off (default)
 *   "multi_tc"      where complex64 multi-target gates on 4-5 targets run:
 *                   2 = on the tensor cores (FP32 operands as TF32 hi + lo
 *                   pairs, three products accumulated in FP32: a few units of
 *                   1e-7 of the largest amplitude per gate), 0 = FP32 on the
 *                   CUDA cores, 1 = by shape (default): 5 targets on the
 *                   tensor cores, 4 on the tensor cores when at least 7
 *                   qubits are neither target nor control (the staged
 *                   kernel) and on the CUDA cores otherwise (paired FP32
 *                   FMAs; through shared-memory tiles when a target is
 *                   below qubit 5)
 *   "multi_tc_stage" tensor-core passes on registers with at least 7 free
 *                   qubits: 1 (default) = staged kernel (tiles copied in
 *                   address order into shared memory two ahead, the A
 *                   operand written to tensor memory, coalesced stores
 *                   whatever the targets); 0 = the register-gather kernel
 *                   (A staged in shared memory; fewer than 7 free qubits
 *                   always use it).  Same products, amplitudes within a
 *                   few units of 1e-7.
 *   "jit"           fused passes of registers of at least "jit_min_qubits"
 *                   stored qubits (default 20) as kernels generated for the
 *                   pass and compiled at run time (NVRTC, sm_103a), cached
 *                   for the process by the pass's structure (coefficients
 *                   are kernel parameters, so other angles reuse them):
 *                   0 = never (the interpreting fused kernel), 1 = compile
 *                   on first use and wait, 2 = compile in the background once
 *                   a pass structure is met a second time, and use the
 *                   interpreting kernel until ready (default: circuits that
 *                   are never rerun cost no compile).  Both
 *                   kernels give bit-identical amplitudes.  Applies to
 *                   complex64 and double-float passes; IEEE-FP64 passes
 *                   only with "jit_fp64" = 1 (they are FP64-pipe bound,
 *                   where the interpreting kernel measured faster).
 *                   "jit_copy": how the generated kernels move tiles between
 *                   HBM and shared memory: 0 = coalesced loads and stores,
 *                   1 = bulk (TMA) copies of the tile's contiguous chunks,
 *                   double-buffered (the next tile's copy overlaps the
 *                   current tile's work; waits bounded, QS_E_TIMEOUT), 2 =
 *                   16-byte async copies (cp.async), double-buffered, -1 =
 *                   by arithmetic (default: 2 for complex64, with tiles of
 *                   2^12 amplitudes, 0 otherwise).  "jit_ctas": resident
 *                   CTAs per SM the generated kernels are built for (1..4,
 *                   0 = by shape, the default: 3 for double-buffered 2^12
 *                   complex64 tiles, else 2).  "jit_direct": 1 (default)
 *                   = the last stage of a generated pass writes its
 *                   amplitudes straight to HBM instead of through shared
 *                   memory (not with bulk copies); 0 = through the tile.
 *                   "jit_swizzle": 1 (default) = the generated kernels
 *                   place a tile's amplitudes in shared memory under an
 *                   XOR swizzle of the 16-byte chunk index (so stages whose
 *                   register bits hold the low positions spread a warp over
 *                   the banks; not with bulk copies, which land chunks
 *                   unpermuted); 0 = plain layout.  Amplitudes are the
 *                   same either way.
 *                   Read-only counters: "jit_launches", "jit_rejected",
 *                   "jit_ready", "jit_pending", "jit_failed",
 *                   "jit_compile_ms".
 *   "plan_cache"    1 (default) = a flush of a gate list that equals one of
 *                   the env's 16 most recently planned lists (same gates and
 *                   parameters, register shape, precision, options, known-
 *                   zero bits and pending scalar) reuses its plan instead of
 *                   planning again; 0 = always plan (and drop the cache).
 *                   Counter: "plan_cache_hits".
 * Unknown keys give QS_E_ARG. */
int setEnvOption(QuESTEnv env, const char *key, int64_t value);
/* getEnvOption: reads an option back, or a counter of the env:
 *   "used_bytes" register memory held, "launches" kernels launched,
 *   "fused_passes" fused-tile passes launched, "fused_vops" vector
 *   operations those passes applied. */
int getEnvOption(QuESTEnv env, const char *key, int64_t *value);
/* setAllocator: device allocations of later registers go through
 * alloc(bytes, ctx) / release(ptr, ctx); null functions restore the built-in
 * cudaMalloc / cudaFree.  alloc must return 256-byte aligned device memory
 * usable on the env's stream, or null on failure (QS_E_NOMEM). */
int setAllocator(QuESTEnv env, void *(*alloc)(size_t bytes, void *ctx),
                 void (*release)(void *ptr, void *ctx), void *ctx);
/* setStream: later work of the env goes to this cudaStream_t (owned by the
 * caller, must outlive its use); null restores the env's own stream.  Queued
 * work is flushed to the old stream first. */
int setStream(QuESTEnv env, void *cudaStream);

/* -------------------------------------------------------------- registers */
/* createQureg: n-qubit state vector (1 <= n <= 36 within memory), returned
 * in |0...0> (Sec. II.B.1: 2^n complex amplitudes; Sec. III: createQureg). */
int createQureg(int numQubits, int precision, QuESTEnv env, Qureg *out);
/* createDensityQureg: N-qubit density matrix held as a 2N-qubit vector
 * (Sec. II.B.1, Eq. 2), returned in |0><0|. */
int createDensityQureg(int numQubits, int precision, QuESTEnv env, Qureg *out);
int destroyQureg(Qureg q);
/* initZeroState: |0...0> (or |0><0|) (Sec. III: initZeroState). */
int initZeroState(Qureg q);
/* initPlusState: |+>^n (or |+><+|^N). */
int initPlusState(Qureg q);
/* copyStateToHost / setAmps: read or write `count` amplitudes starting at
 * flat index `start` (direct amplitude access, Sec. II.B.1).  For a
 * density matrix the flat index is j + 2^N k.  QS_C64 registers are
 * converted to / from double. */
int copyStateToHost(Qureg q, Complex *dst, int64_t start, int64_t count);
int setAmps(Qureg q, const Complex *src, int64_t start, int64_t count);
int getNumQubits(Qureg q, int *out);
int getNumAmps(Qureg q, int64_t *out);
/* getQuregInfo: any output pointer may be null.  devicePtr is the register's
 * amplitude array (valid until destroyQureg; the caller must sync first).
 * The caller may write amplitudes through it: asking for it makes the
 * library drop what it knows about the register's contents. */
int getQuregInfo(Qureg q, int *numQubits, int *isDensity, int *precision,
                 void **devicePtr);

/* ------------------------------------------------------------------ gates */
/* Single-target gates: the pass of Eq. 1 over amplitude pairs differing in
 * bit `target`.  On a density matrix each is applied as U rho U^dagger
 * (Eq. 2). */
int hadamard(Qureg q, int target);
int pauliX(Qureg q, int target);
int sqrtX(Qureg q, int target);     /* [[1+i, 1-i], [1-i, 1+i]] / 2          */
int sqrtY(Qureg q, int target);     /* (1+i)/2 [[1, -1], [1, 1]]              */
int tGate(Qureg q, int target);     /* diag(1, exp(i pi/4)), the pi/8 gate    */
int phaseShift(Qureg q, int target, double angle);  /* diag(1, exp(i angle)) */
/* compactUnitary: [[alpha, -conj(beta)], [beta, conj(alpha)]] with
 * |alpha|^2 + |beta|^2 = 1 (within 1e-10, else QS_E_UNITARY). */
int compactUnitary(Qureg q, int target, Complex alpha, Complex beta);
/* unitary: any 2x2 unitary (max |U U^dagger - I| <= 1e-10). */
int unitary(Qureg q, int target, ComplexMatrix2 u);
/* Controlled gates (Eq. 1 generalised to control bits, Sec. II.B.1): the
 * pair update happens only where every control bit is 1. */
int controlledNot(Qureg q, int control, int target);
int controlledUnitary(Qureg q, int control, int target, ComplexMatrix2 u);
int multiControlledUnitary(Qureg q, const int *controls, int numControls,
                           int target, ComplexMatrix2 u);
/* Multi-target gates: a dense 2^m x 2^m unitary on m = numTargets qubits
 * (1..5), the block of 2^m amplitudes differing in the target bits taking
 * the place of Eq. 1's pair; the paper notes the density-matrix rule of
 * Eq. 2 holds also for multi-qubit gates (Sec. II.B.1).  Bit k of the
 * matrix's row / column index is qubit targets[k] (targets[0] is the least
 * significant).  `u` is row-major (u[row * 2^m + column]), copied at call
 * time, unitary within 1e-10 (QS_E_UNITARY otherwise).  Targets and
 * controls must be distinct (QS_E_DUP).  These gates run as their own pass;
 * queued single-target gates before and after them are fused as usual. */
int multiQubitUnitary(Qureg q, const int *targets, int numTargets, const Complex *u);
int multiControlledMultiQubitUnitary(Qureg q, const int *controls, int numControls,
                                     const int *targets, int numTargets, const Complex *u);
/* twoQubitUnitary: u.m[row][column], bit 0 of the index is target1. */
int twoQubitUnitary(Qureg q, int target1, int target2, ComplexMatrix4 u);
/* controlledPhaseFlip (CZ): negates amplitudes with both bits set. */
int controlledPhaseFlip(Qureg q, int qubit1, int qubit2);
/* multiControlledPhaseFlip: negates amplitudes whose index has every listed
 * bit set (1 <= numControls <= numQubits). */
int multiControlledPhaseFlip(Qureg q, const int *controls, int numControls);

/* --------------------------------------------------------------- channels */
/* Density matrices only (QS_E_NOT_DENSITY otherwise).  The paper names
 * dephasing and depolarising noise (abstract; Sec. II.B.1) without formulas;
 * this library's reading:
 *   mixDephasing(p):    rho -> (1-p) rho + p Z rho Z,  0 <= p <= 1/2
 *   mixDepolarising(p): rho -> (1-p) rho + p/3 (X rho X + Y rho Y + Z rho Z),
 *                       0 <= p <= 3/4 */
int mixDephasing(Qureg q, int target, double prob);
int mixDepolarising(Qureg q, int target, double prob);

/* ------------------------------------------------------------- reductions */
/* Results are accumulated in FP64 on the GPU in a fixed order (repeatable
 * bit for bit on one GPU).  State vector: sum |a|^2; density matrix: the
 * trace sum_j Re rho[j][j]. */
int calcTotalProb(Qureg q, double *out);
/* Probability that `qubit` reads `outcome` (0 or 1). */
int calcProbOfOutcome(Qureg q, int qubit, int outcome, double *out);
/* collapseToOutcome: projects `qubit` onto `outcome` and renormalises (scale
 * 1/sqrt(p), or 1/p for a density matrix, in FP64).  Writes p to probOut
 * (may be null).  p < 1e-13 (QS_C128) or 1e-6 (QS_C64) gives
 * QS_E_ZERO_PROB and leaves the register unchanged. */
int collapseToOutcome(Qureg q, int qubit, int outcome, double *probOut);
/* calcPurity: Tr(rho^2) = sum_n |rho'_n|^2 of a density matrix. */
int calcPurity(Qureg q, double *out);
/* calcInnerProduct: <bra|ket> = sum_j conj(bra_j) ket_j, accumulated in FP64
 * (complex64 amplitudes widened first), for two state vectors of the same
 * qubit count and either precision (QuEST's API call of this name; the
 * paper's Sec. III lists the API's measurement calls).  Both registers'
 * queued gates are applied first; the reduction runs on bra's environment
 * stream after ket's environment stream is synchronised.  Errors:
 * QS_E_NOT_DENSITY for a density matrix, QS_E_QUBIT for unequal sizes. */
int calcInnerProduct(Qureg bra, Qureg ket, Complex *out);
/* calcFidelity: |<a|b>|^2 of two state vectors (as calcInnerProduct; no
 * renormalisation: divide by both calcTotalProb for the fidelity of the
 * normalised states). */
int calcFidelity(Qureg a, Qureg b, double *out);

/* ------------------------------------------------------------ bulk calls */
/* One operation of a gate list; the same operations as the calls above. */
enum {
    QS_OP_H = 1, QS_OP_X = 2, QS_OP_SQRTX = 3, QS_OP_SQRTY = 4, QS_OP_T = 5,
    QS_OP_PHASE = 6,        /* params[0] = angle                               */
    QS_OP_COMPACT = 7,      /* params = alpha.re, alpha.im, beta.re, beta.im   */
    QS_OP_UNITARY = 8,      /* params = u00 u01 u10 u11 as (re, im)            */
    QS_OP_CNOT = 9,         /* controls[0], target                             */
    QS_OP_CUNITARY = 10,    /* controls[0..numControls), target, params as U   */
    QS_OP_CZ = 11,          /* target and target2                              */
    QS_OP_MCPF = 12,        /* controls[0..numControls)                        */
    QS_OP_DEPHASE = 13,     /* target, params[0] = p                           */
    QS_OP_DEPOL = 14        /* target, params[0] = p                           */
};
#define QS_MAX_OP_CONTROLS 8
typedef struct {
    int32_t kind;
    int32_t target;
    int32_t target2;
    int32_t numControls;
    int32_t controls[QS_MAX_OP_CONTROLS];
    double params[8];
} QSOp;

/* applyCircuit: validates every op first (QS_E_* naming the first bad op's
 * index in qsLastError, nothing applied), then applies them in order, as if
 * by the individual calls. */
int applyCircuit(Qureg q, const QSOp *ops, int64_t numOps);

/* ------------------------------------------------------------- batches */
/* Many independent state vectors advanced together (a batched form of the
 * per-gate pass of Eq. 1; the paper runs one register at a time).
 * createBatch: takes `count` distinct state-vector registers of one env and
 * one precision (each >= 4 qubits for QS_C128, >= 5 for QS_C64) with their
 * queued gates, which it consumes.  Each register is planned into fused
 * passes exactly as a single-register flush would plan it (tile size
 * tileQubits, 0 = default), the passes of all registers are grouped into
 * waves (wave w = pass w of every register), and the launches plus one FP64
 * norm per register are captured into a CUDA graph on the env's stream.
 * One replay (runBatch) starts every register from |0...0> and applies its
 * whole circuit; registers of up to 2^k amplitudes never leave shared memory
 * within a pass.  The registers must outlive the batch; their amplitudes
 * after a replay are read with copyStateToHost as usual.
 * runBatch: queues one replay (asynchronous).
 * getBatchNorms: waits, then writes count doubles: sum |a|^2 per register
 *   after the last replay, accumulated in FP64.
 * getBatchInfo: tile size requested (0 = default), total passes, waves,
 *   algorithmic bytes and flops of one replay (any pointer may be null).
 * tuneBatch: autotuner: re-plans and times `replays` replays for every
 *   candidate tile size (5..13), keeps the fastest; writes it to *chosen.
 *   A tile has at least 2^(R+5) amplitudes where the register has as many
 *   (R = 5 register bits for QS_C64, 4 for QS_C128), so candidates below
 *   R + 5 act as R + 5 on such registers and as the register itself on
 *   smaller ones.
 * tuneBatchJoint: the same over every pair of a candidate tile size and a
 *   candidate fusion depth (the cap on operations per fused pass, 0 = the
 *   planner's default, else 1..256); writes the fastest pair.
 * destroyBatch: frees the batch (not the registers). */
typedef struct { int64_t id; } QSBatch;
int createBatch(QuESTEnv env, const Qureg *regs, int count, int tileQubits, QSBatch *out);
int runBatch(QSBatch batch);
int getBatchNorms(QSBatch batch, double *out);
int getBatchInfo(QSBatch batch, int *tileQubits, int64_t *passes, int *waves, double *bytes,
                 double *flops);
int tuneBatch(QSBatch batch, const int *candidates, int numCandidates, int replays, int *chosen);
int tuneBatchJoint(QSBatch batch, const int *tileCandidates, int numTile, const int *depthCandidates,
                   int numDepth, int replays, int *chosenTile, int *chosenDepth);
int destroyBatch(QSBatch batch);

/* ------------------------------------------------------------- serving */
/* A request loop: circuits submitted at any time run as soon as a slot and
 * memory are free, concurrently with the ones already on the GPU (the paper
 * runs one circuit per process; this is a library extension).
 * serveCreate: `slots` execution slots (1..64), each with its own CUDA
 *   stream and scratch; registers live within `budgetBytes` (2^n x 8 or 16
 *   bytes each, density matrices 2^(2N)); `fusion` as the env option.  A
 *   scheduler thread admits requests in arrival order while a slot is free
 *   and the next request fits the budget.  Register memory comes from the
 *   device's stream-ordered pool (its release threshold is raised so freed
 *   blocks stay cached).  complex128 arithmetic and tile size follow the
 *   env's options at creation.
 * serveSubmit: validates and queues one request, returns its ticket.  The
 *   op list is copied; outAmps (optional host buffer for the first outCount
 *   final amplitudes, flat index as copyStateToHost) must stay valid until
 *   the result is collected.  A request larger than the budget gives
 *   QS_E_NOMEM; an invalid circuit gives its QS_E_* code (nothing queued).
 * servePoll: waits up to timeoutUs microseconds for the ticket's result;
 *   QS_E_TIMEOUT if it is not finished (the ticket stays valid), otherwise
 *   fills *out and retires the ticket.
 * serveSetOption: admission policy past saturation (both 0 = none, the
 *   default: every request is queued until it runs, so latency grows without
 *   bound once arrivals outpace the GPU):
 *     "max_queue"     back-pressure: serveSubmit refuses a request with
 *                     QS_E_BUSY (nothing queued) while this many wait;
 *     "max_queue_us"  shedding: a request that has waited this long without
 *                     being admitted is dropped; its result has status
 *                     QS_E_BUSY.  Admitted requests then wait at most about
 *                     this long (the scheduler checks every 50 ms at most).
 *   Counters (serveGetOption): "queued", "shed", "refused".
 * serveDestroy: stops admitting, waits for the requests on the GPU, cancels
 *   the queued ones, frees the slots. */
typedef struct { int64_t id; } QSServer;
typedef struct {
    int32_t isDensity;      /* 0: state vector, 1: density matrix            */
    int32_t precision;      /* QS_C64 or QS_C128                             */
    int32_t numQubits;
    int32_t measureQubit;   /* qubit whose outcome-0 probability is returned */
    const QSOp *ops;
    int64_t numOps;
    Complex *outAmps;       /* optional, may be null                         */
    int64_t outCount;
} QSRequest;
typedef struct {
    int32_t status;         /* QS_OK or the request's error                  */
    int32_t slot;           /* slot that ran it                              */
    double totalProb;       /* calcTotalProb of the final state (FP64)       */
    double probOutcome0;    /* calcProbOfOutcome(measureQubit, 0)            */
    double queuedUs;        /* submit -> admitted                            */
    double latencyUs;       /* submit -> results ready                       */
} QSResult;
int serveCreate(QuESTEnv env, int slots, int64_t budgetBytes, int fusion, QSServer *out);
int serveSubmit(QSServer server, const QSRequest *req, int64_t *ticket);
int servePoll(QSServer server, int64_t ticket, QSResult *out, int64_t timeoutUs);
int serveSetOption(QSServer server, const char *key, int64_t value);
int serveGetOption(QSServer server, const char *key, int64_t *value);
int serveDestroy(QSServer server);

/* ------------------------------------------------ partitioned registers */
/* The paper's distributed state vector (Sec. II.B.2): an n-qubit state vector
 * split into P = 2^k parts of 2^(n-k) amplitudes by its top k index bits (in
 * the paper, one part per node).  Gates that move amplitudes along a qubit
 * held in the part index ("global") need other parts' amplitudes; the paper
 * exchanges whole parts between pairs of nodes.  Here a global qubit about
 * to be moved is first swapped with a local one (each pair of parts
 * differing in that bit exchanges half of its amplitudes through send and
 * receive buffers), after which the gate, and the fused tiles that follow,
 * run inside every part; the qubit map is kept.  Diagonal gates and
 * controls on global qubits need no exchange (a part knows its global
 * bits).  In this library all parts live on the env's GPU and the exchange
 * is a device-to-device copy between the buffers, the step a deployment
 * with one part per GPU would carry out as point-to-point transfers; the
 * swap schedule and the reductions are the same.
 * createPartitionedQureg: numQubits 2..40, globalQubits k 1..min(6, n-1)
 *   (P = 2^k parts), QS_C64 / QS_C128; starts in |0...0>.  Memory: the
 *   parts plus four half-part buffers.
 * partApplyCircuit: single-target gates, controlled gates, phases and sign
 *   flips (QS_OP_H .. QS_OP_MCPF; channels and multi-target gates give
 *   QS_E_ARG), validated as applyCircuit does; queued like applyCircuit,
 *   with swaps where the schedule needs them.
 * partCalcTotalProb / partCalcProbOfOutcome: each part reduces in FP64, the
 *   part sums add in part order (the all-reduce of a distributed run).
 * partCopyStateToHost: the whole 2^n state in logical index order (the
 *   qubit map undone), into dst (caller-owned, 2^n Complex).
 * partGetInfo: sizes, the logical -> physical qubit map (n ints), swaps run
 *   and bytes exchanged between parts so far (any pointer may be null).
 * partPlanSchedule (host only, no GPU): the schedule partApplyCircuit runs
 *   for ops on a fresh register: steps of kind 0 (apply op `op` in every
 *   part) or 1 (swap physical global position globalPos with local position
 *   localPos), and the final qubit map; maxSteps 0 only counts. */
typedef struct { int64_t id; } QSPartReg;
typedef struct {
    int32_t kind;       /* 0: local op, 1: qubit swap        */
    int32_t op;         /* kind 0: index into the op list    */
    int32_t globalPos;  /* kind 1: physical position >= n-k  */
    int32_t localPos;   /* kind 1: physical position < n-k   */
} QSPartStep;
int createPartitionedQureg(int numQubits, int globalQubits, int precision, QuESTEnv env, QSPartReg *out);
int destroyPartitionedQureg(QSPartReg reg);
int partApplyCircuit(QSPartReg reg, const QSOp *ops, int64_t numOps);
int partCalcTotalProb(QSPartReg reg, double *out);
int partCalcProbOfOutcome(QSPartReg reg, int qubit, int outcome, double *out);
int partCopyStateToHost(QSPartReg reg, Complex *dst);
int partGetInfo(QSPartReg reg, int *numQubits, int *globalQubits, int *perm, int64_t *swaps,
                double *exchangedBytes);
int partPlanSchedule(int numQubits, int globalQubits, const QSOp *ops, int64_t numOps, QSPartStep *steps,
                     int64_t maxSteps, int64_t *numSteps, int *finalPerm);

/* ------------------------------------------------- allocation-free norm */
/* calcTotalProbNoAlloc: sum over j of |amps[j]|^2 in FP64, for callers that
 * cannot allocate device memory (a host framework that owns the whole device
 * through its own pool, a plug-in handed fixed buffers, code that must not
 * trigger an allocation's implicit synchronisation).  It needs no
 * environment and calls no allocator: its scratch is a fixed array of 65536
 * doubles (512 KiB) in the library's own device memory, held by every GPU
 * that loads the library until the process exits.  The paper has no
 * counterpart; this is a library convenience.
 *   amps       device pointer to numAmps interleaved complex amplitudes
 *              (double2 for QS_C128, float2 for QS_C64), owned by the caller,
 *              aligned to one amplitude (16 / 8 bytes; else QS_E_ARG).  For a
 *              state vector the result is the total probability; for a
 *              density matrix's 2^(2N) stored entries it is the purity
 *              Tr rho^2, not the trace (use calcTotalProb for Tr rho)
 *   precision  QS_C64 or QS_C128
 *   numAmps    1 .. 2^30 (one scratch slot per 16384 amplitudes); larger
 *              arrays are rejected with QS_E_ARG and a message
 *   out        device pointer to one double, owned by the caller, 8-byte
 *              aligned (else QS_E_ARG); written when the call's kernels run
 *   stream     cudaStream_t the work is queued on (null = legacy default);
 *              the call returns without waiting
 * The first call on a device looks up the scratch array's device address
 * with that device current; make that first call before any stream capture.
 * The address is kept until the process exits: after cudaDeviceReset on a
 * device, do not call this entry point on that device again.  A CUDA error
 * left pending by earlier work is reported (QS_E_CUDA) without being cleared,
 * and nothing is launched.
 * All calls share the one scratch array: calls whose kernels overlap on the
 * GPU (different streams, or several host threads) race and give wrong
 * sums; serialise them.  Every scratch slot a call reads is written by that
 * call first, so stale contents from earlier calls do not matter.  The
 * result equals calcTotalProb's up to FP64 summation order. */
int calcTotalProbNoAlloc(const void *amps, int precision, int64_t numAmps, double *out,
                         void *stream);

/* ---------------------------------------------------------- kernel stats */
/* Per-kernel-class timing, for roofline reporting.  With option "profile"
 * set to 1, every kernel launch of the env is bracketed by CUDA events on
 * the env's stream and charged to its class (a name such as
 * "sv_pair_gen_c128").  getKernelStats waits for the stream, then fills up
 * to maxOut entries and writes the number of classes to *count.  Bytes and
 * flops are algorithmic: the amplitudes a launch must read and write and
 * the floating-point operations its arithmetic needs (FMA = 2).  alu_ops
 * (fused passes and batches; 0 elsewhere) counts the arithmetic
 * instructions that arithmetic issues, each add, multiply or FMA once, in
 * the kernel's own precision (double-float counted in FP32 instructions). */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
    double bytes;
    double flops;
    double alu_ops;
} QSKernelStat;
int getKernelStats(QuESTEnv env, QSKernelStat *out, int maxOut, int *count);
int resetKernelStats(QuESTEnv env);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_H */
