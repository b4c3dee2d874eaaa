/*
 * spx.h - C ABI of the B300 device-scheduled STF tile-task library.
 *
 * The library runs a sequential-task-flow (STF) graph of tile tasks on one
 * GPU.  A single host thread inserts tasks with their data accesses; the
 * library derives the dependencies on the device (successor CSR + in-degree
 * counters in HBM) and executes the graph in one persistent kernel whose CTAs
 * pop ready tasks from a device work queue, run the tile operation and
 * release the successors.  Model: Specx, arXiv 2308.15964, section "Task graph
 * description" (task graph object, task insertion with SpRead / SpWrite /
 * SpCommutativeWrite, priorities) and section "Internal implementation"
 * (address-keyed data handles with ordered dependency lists).  The tile
 * operations are the four task types of the paper's tiled Cholesky (section
 * "Numerical applications": POTRF, TRSM, SYRK, GEMM), the tiled GEMM whose
 * tasks depend on the blocks of C, and the block triangular solves.
 *
 * Conventions for every call:
 *   - Return value: SPX_OK (0) on success, SPX_NOT_SPD (1) when a POTRF met a
 *     non-positive pivot, a negative SPX_ERR_* code otherwise.  A failing call
 *     leaves the graph unchanged unless stated.
 *   - Pointers named dev_* are CUDA device pointers; every other pointer is a
 *     host pointer.  Streams are cudaStream_t passed as void*.
 *   - Matrices are row-major FP64 unless a dtype says otherwise: element
 *     (r, c) of a tile with leading dimension ld is at ptr[r*ld + c].
 *   - Ownership: the caller owns all tile memory and must keep it alive and
 *     untouched by other work until spx_graph_wait returns (paper, section
 *     "Task insertion": objects must outlive the tasks that use them).  The
 *     graph owns its own metadata (host and device arrays).
 *   - Not thread-safe per graph: one host thread drives a graph.
 */
#ifndef SPX_H_
#define SPX_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spx_graph* spx_graph_t;

/* Access modes (paper, section "Task insertion").
 *   SPX_READ               the task only reads the data.
 *   SPX_WRITE              the task reads and/or writes; ordered and exclusive.
 *   SPX_COMMUTATIVE_WRITE  reads and writes, but the tasks of one run of
 *                          commutative writes inserted one after another may
 *                          execute in any order, one at a time.
 *   SPX_ATOMIC_WRITE       reads and writes, the task protecting its own
 *                          updates: ordered like a READ (a run of atomic
 *                          writes inserted one after another forms one group
 *                          whose members may run at the same time; accesses
 *                          of other modes before and after the run are
 *                          ordered with it).  The tile ops that accept it
 *                          (GEMM_NN_ADD and AXPY on the written operand)
 *                          then add into the tile with atomic additions, in
 *                          an order that varies from run to run.
 *   SPX_MAYBE_WRITE        the task may or may not write.  The paper attaches
 *                          speculative execution to it; this library does not
 *                          speculate, so it is ordered exactly like a WRITE.
 * A task that names the same tile twice gets the merged mode: the mode when
 * both agree (READ+READ = READ, COMM+COMM = COMM, ATOMIC+ATOMIC = ATOMIC,
 * MAYBE+MAYBE = MAYBE), WRITE otherwise. */
enum {
  SPX_READ = 0,
  SPX_WRITE = 1,
  SPX_COMMUTATIVE_WRITE = 2,
  SPX_ATOMIC_WRITE = 3,
  SPX_MAYBE_WRITE = 4
};

/* Tile operations.  Operand order (the handles[] of spx_task_insert) and the
 * required access mode of each operand are fixed per op:
 *   SPX_OP_POTRF        (A_kk:W)                A_kk = L L^T, lower L written
 *                                               over the lower triangle; the
 *                                               strict upper triangle is kept.
 *   SPX_OP_TRSM         (L_kk:R, A_ik:W)        A_ik <- A_ik L_kk^{-T}
 *   SPX_OP_SYRK         (L_ik:R, A_ii:W)        A_ii <- A_ii - L_ik L_ik^T
 *                                               (lower triangle only)
 *   SPX_OP_GEMM_NT_SUB  (L_ik:R, L_jk:R, A_ij:W) A_ij <- A_ij - L_ik L_jk^T
 *   SPX_OP_GEMM_NN_ADD  (A_ik:R, B_kj:R, C_ij:W|C) C_ij <- C_ij + A_ik B_kj
 *   SPX_OP_TRSM_L_FWD   (L_kk:R, X_k:W)         X_k <- L_kk^{-1} X_k
 *   SPX_OP_GEMM_FWD     (L_ik:R, X_k:R, X_i:W)  X_i <- X_i - L_ik X_k
 *   SPX_OP_TRSM_LT_BWD  (L_kk:R, X_k:W)         X_k <- L_kk^{-T} X_k
 *   SPX_OP_GEMM_BWD     (L_ki:R, X_k:R, X_i:W)  X_i <- X_i - L_ki^T X_k
 *   SPX_OP_NOP          any handles, any modes  does nothing (graph tests)
 *   SPX_OP_SPIN         any handles, any modes  busy-waits arg nanoseconds
 *   SPX_OP_COPY         (X:R, Y:W)              Y <- X (same shape)
 *   SPX_OP_AXPY         (X:R, Y:W)              Y <- Y + alpha X (same shape;
 *                                               alpha from spx_task_set_scalar,
 *                                               default 1; computed as
 *                                               fl(fl(alpha x) + y) in Y's
 *                                               type, one rounding when
 *                                               alpha = 1)
 *   SPX_OP_TRMM         (T:R, X:R, Y:W)         Y <- T X (arg 0) or T^T X
 *                                               (arg 1); T square, lower
 *                                               triangular: its entries above
 *                                               the diagonal must be zero (as
 *                                               TRTRI leaves them); X and Y
 *                                               distinct tiles
 *   SPX_OP_TRTRI        (L_kk:R, V_k:W)         V_k <- L_kk^{-1} (lower
 *                                               triangle of L_kk; V_k square,
 *                                               written whole, zero above its
 *                                               diagonal)
 *   SPX_OP_POTRF_PANEL  (A_kk:W, A_ik:W)        POTRF of A_kk and the solve
 *                                               A_ik <- A_ik L_kk^{-T} in one
 *                                               task: the rows of A_ik join the
 *                                               panel rows of each 64-column
 *                                               step (the same arithmetic as
 *                                               POTRF then TRSM, fewer phase
 *                                               boundaries on the critical
 *                                               path); A_ik.cols = A_kk.cols.
 *                                               prec SPX_F64, or SPX_F64_OZAKI
 *                                               to split A_ik at the end
 *   SPX_OP_SPLIT        (X:W)                   split X (FP64) into the split
 *                                               slot of its tile: row r gets
 *                                               its own exponent, K = X's
 *                                               columns (the A operand of a
 *                                               split product); X's FP64
 *                                               entries are not changed.
 *                                               prec SPX_F64_OZAKI only
 *   SPX_OP_SPLIT_T      (X:W)                   split X^T into the slot: slot
 *                                               row c is column c of X with
 *                                               its own exponent, K = X's
 *                                               rows (the B operand of C +=
 *                                               A X).  prec SPX_F64_OZAKI only
 *   SPX_OP_NBODY_SELF   (P:W)                   interactions of the particles
 *                                               of group P with each other
 *   SPX_OP_NBODY_PAIR   (P:W, Q:W)              interactions between groups P
 *                                               and Q (both updated)
 *                       A particle group is an n x 8 FP64 tile, one particle
 *                       per row: x, y, z, charge q, then the accumulated
 *                       potential phi and field E (3 components).  Each
 *                       interaction of target i with source j (j != i) adds
 *                       q_j / r to phi_i and q_j (x_i - x_j) / r^3 to E_i,
 *                       r = |x_i - x_j| (the paper's particle test case: a
 *                       direct Coulomb summation, about 17 flops and one
 *                       square root per interaction, section "Numerical
 *                       applications"); coincident particles (r = 0) do not
 *                       interact.
 *   SPX_OP_TRSM_INV     (V_kk:R, A_ik:W)        A_ik <- A_ik V_kk^T with V_kk
 *                                               = L_kk^{-1} from TRTRI (lower,
 *                                               zero above the diagonal): the
 *                                               TRSM of the mixed-precision
 *                                               factorization as a product on
 *                                               the tensor cores; prec
 *                                               SPX_TF32 / SPX_BF16 /
 *                                               SPX_F64_OZAKI only (see the
 *                                               prec enum), A_ik.cols a
 *                                               multiple of 32
 * GEMM_NN_ADD with prec SPX_F64_OZAKI forms C_ij + A_ik B_kj as a split
 * product on the tensor cores from A_ik's slot (written by SPLIT) and B_kj's
 * slot (written by SPLIT_T), one rounding per task and entry; C_ij by WRITE
 * or COMMUTATIVE_WRITE (not ATOMIC_WRITE).
 * Operand element types: SPX_DT_F64 throughout, except that GEMM_FWD,
 * GEMM_BWD and TRMM also take all three operands SPX_DT_F32 (FP32
 * arithmetic) when the written tile has at most 16 columns, and COPY / AXPY
 * take X and Y each SPX_DT_F64 or SPX_DT_F32 (FP64 -> FP32 rounds to
 * nearest, FP32 -> FP64 is exact); anything else is SPX_ERR_INVALID_ARG.
 * A write operand may also be given as SPX_COMMUTATIVE_WRITE; such tasks
 * run as one part and take per-tile locks in ascending handle order (the
 * paper locks data handles sorted by address, section "Internal
 * implementation").  SPX_MAYBE_WRITE is accepted wherever SPX_WRITE is;
 * SPX_ATOMIC_WRITE only on the written operand of GEMM_NN_ADD and AXPY (and
 * by NOP / SPIN). */
enum {
  SPX_OP_POTRF = 0,
  SPX_OP_TRSM = 1,
  SPX_OP_SYRK = 2,
  SPX_OP_GEMM_NT_SUB = 3,
  SPX_OP_GEMM_NN_ADD = 4,
  SPX_OP_TRSM_L_FWD = 5,
  SPX_OP_GEMM_FWD = 6,
  SPX_OP_TRSM_LT_BWD = 7,
  SPX_OP_GEMM_BWD = 8,
  SPX_OP_NOP = 9,
  SPX_OP_SPIN = 10,
  SPX_OP_COPY = 11,
  SPX_OP_AXPY = 12,
  SPX_OP_TRMM = 13,
  SPX_OP_TRTRI = 14,
  SPX_OP_TRSM_INV = 15,
  SPX_OP_NBODY_SELF = 16,
  SPX_OP_NBODY_PAIR = 17,
  SPX_OP_POTRF_PANEL = 18,
  SPX_OP_SPLIT = 19,
  SPX_OP_SPLIT_T = 20,
  SPX_NUM_OPS = 21
};

/* Arithmetic of a task.  SPX_F64: FP64 throughout.  SPX_TF32 / SPX_BF16
 * (mixed precision; allowed for TRSM, TRSM_INV, SYRK and GEMM_NT_SUB): SYRK
 * and GEMM_NT_SUB compute the product of the low-precision copies of their
 * factor operands on the tensor cores with FP32 accumulation and subtract it
 * from the FP64 output tile; TRSM solves in FP64 and then writes the
 * low-precision copy of its result (round to nearest; TF32 as FP32 with the
 * low 13 mantissa bits cleared).  TRSM_INV (either prec) forms A_ik V_kk^T
 * on the tensor cores from split operands: every FP64 entry x is split into
 * TF32 parts hi + lo (hi = x rounded to TF32, lo = the rest rounded to
 * TF32; |x - hi - lo| <= about 2^-22 |x|) and the three products
 * hi*hi + hi*lo + lo*hi accumulate in FP32 (the lo*lo term, about 2^-22
 * relative, is dropped), i.e. about FP32 accuracy; the FP64 tile receives
 * the accumulator widened exactly and the low-precision copy its rounding
 * to the task's type.
 * SPX_F64_OZAKI (the split scheme of Ozaki, Ogita, Oishi and Rump, 2012;
 * one-CTA-per-SM kernel): a split operand keeps, per row, the exponent e_r
 * (the smallest e >= -1022 with every |a_rk| < 2^e) and the integer X_rk =
 * a_rk 2^(55 - e_r) rounded to nearest even, as eight balanced base-128
 * digits stored as BF16 in the tile's split slot (SPLIT, SPLIT_T, or the
 * last phase of TRSM / TRTRI / TRSM_INV / POTRF_PANEL writes it).  A split
 * product sums the digit products of planes s + t <= 7 on the tensor cores
 * in FP32 (every partial sum an integer below 2^24, so exact for K <= 512),
 * joins them in 64-bit integers and rounds once to FP64: per entry the error
 * is at most K 9.05 2^-56 2^(e_r + f_c) before the final rounding, the
 * accuracy of an FP64 dot product.  SYRK and GEMM_NT_SUB subtract the
 * product, GEMM_NN_ADD adds it, TRSM_INV stores it. */
enum { SPX_F64 = 0, SPX_TF32 = 1, SPX_BF16 = 2, SPX_F64_OZAKI = 3 };

/* SPX_F64_OZAKI: FP64 products emulated on the BF16 tensor cores by splitting
 * (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 2012),
 * allowed for TRSM, SYRK and GEMM_NT_SUB whose factor tiles have split slots
 * in a store registered with spx_ozaki_register.  The paper's Cholesky spends
 * almost all of its flops in these trailing updates (section "Numerical
 * applications"); on this GPU the FP64 SIMT pipe peaks at about 1.2 TFLOP/s
 * while the BF16 tensor cores reach about 2 PFLOP/s.
 *   TRSM solves in FP64 and then splits its result: per row r, with e_r the
 *   smallest integer such that every |a_rk| < 2^e_r (-1022 for a zero row),
 *   X_rk = a_rk 2^(55 - e_r) rounded to the nearest integer (ties to even)
 *   is written as eight balanced base-128 digits, X = sum_s sigma_s 128^(7-s)
 *   (sigma_1..7 in [-64, 63] from the bottom, sigma_0 in [-64, 64]), each
 *   stored exactly as a BF16; e_r is stored beside them.
 *   SYRK / GEMM_NT_SUB (C -= A B^T, K = the factor tiles' columns <= 512)
 *   accumulate P_d = sum over s + t = d of sigma_s(A) tau_t(B)^T for
 *   d = 0..7 in separate FP32 accumulators on the tensor cores (pairs with
 *   s + t > 7 are dropped).  |sigma tau| <= 2^12 and K <= 512 bound every
 *   |P_d| by 2^24, so each P_d is an exact integer.  With
 *   F = sum_d P_d 128^(7-d) (formed exactly in integers), the entry becomes
 *   C_rc - v with v = F 2^(e_r + f_c - 61) rounded once to FP64 and the
 *   subtraction rounded once.  Error of v against the exact product of the
 *   FP64 tiles: at most about 2^-52.8 * K * 2^(e_r + f_c) (the input rounding
 *   and the dropped pairs), below the worst-case bound of an FP64 dot
 *   product of length K.  Finite inputs; products whose scale leaves the FP64
 *   normal range are rounded twice. */

/* Element type of a registered tile. */
enum { SPX_DT_F64 = 0, SPX_DT_F32 = 1, SPX_DT_BF16 = 2 };

/* Executors.  SPX_EXEC_PERSISTENT is the product: one persistent kernel with a
 * device work queue.  SPX_EXEC_PER_TASK is the comparison baseline: one kernel
 * launch per task, on the given stream, in insertion order (a valid
 * topological order of any STF graph), running the same tile code.
 * SPX_EXEC_STREAMS is a second baseline after the paper's GPU set-up (four
 * streams per GPU, section "Numerical Applications"): the same per-task
 * launches in insertion order, round-robin over four streams, with one event
 * wait per predecessor that ran on another stream (the DAG is derived on the
 * device and read back once); tasks with a commutative write all go to the
 * first stream, so the members of a commutative run never overlap.
 * cfg.cuda_graph is ignored for it. */
enum { SPX_EXEC_PERSISTENT = 0, SPX_EXEC_PER_TASK = 1, SPX_EXEC_STREAMS = 2 };

/* Status codes. */
enum {
  SPX_OK = 0,
  SPX_NOT_SPD = 1,            /* a POTRF pivot was <= 0 or NaN; info = column */
  SPX_ERR_INVALID_ARG = -1,   /* bad pointer, size, op, mode or operand shape */
  SPX_ERR_BAD_HANDLE = -2,    /* unknown tile handle or task id */
  SPX_ERR_STATE = -3,         /* call not allowed in the graph's state */
  SPX_ERR_OOM = -4,           /* host or device allocation failed */
  SPX_ERR_QUEUE_FULL = -5,    /* device work queue capacity exceeded */
  SPX_ERR_TIMEOUT = -6,       /* device watchdog or host wait timeout */
  SPX_ERR_CUDA = -7,          /* a CUDA runtime call failed */
  SPX_ERR_BAD_OP = -8,        /* device met an unknown op (corrupt graph) */
  SPX_ERR_NO_DEVICE = -9      /* no usable CUDA device */
};

/* Graph configuration.  Zero fields take defaults. */
typedef struct {
  int num_ctas;               /* persistent CTAs; 0 = resident maximum        */
  int executor;               /* SPX_EXEC_*                                   */
  int trace;                  /* 1 = record per-task timestamps and SM ids    */
  int no_split;               /* 1 = run every task as a single part          */
  unsigned long long watchdog_ns; /* device gives up after this long without
                                 finishing a task part; 0 = 10 s              */
  long long queue_capacity;   /* entries per priority queue; 0 = exact size   */
  int cuda_graph;             /* 1 = capture the re-execution sequence of a
                                 reset graph (state reset, queue set-up,
                                 executor, status copy) into a CUDA graph on
                                 its second execute and replay it after     */
  int priorities;             /* 0 = the priorities given at insertion;
                                 1 = from the critical path of the DAG (see
                                 spx_graph_assign_priorities), at the first
                                 execute                                      */
} spx_graph_config_t;

/* Fill *cfg with the defaults. */
void spx_config_default(spx_graph_config_t* cfg);

/* Create an empty graph (paper, section "Task graph description": the task
 * graph object is separate from the engine that runs it).  cfg may be NULL.
 * No device memory is touched until the first execute/derive.
 * Errors: SPX_ERR_INVALID_ARG (out NULL or bad cfg), SPX_ERR_OOM. */
int spx_graph_create(spx_graph_t* out, const spx_graph_config_t* cfg);

/* Register a tile (a data object of the STF model) and get its handle.
 *   dev_ptr  device address of element (0,0); it is also the dependency key
 *            (paper, section "Internal implementation": the address of the
 *            object is the key of its data handle).  Registering the same
 *            address again returns the same handle when rows/cols/ld/dtype
 *            agree, SPX_ERR_INVALID_ARG otherwise.  Overlapping tiles with
 *            different addresses are distinct handles (not detected).
 *   rows, cols >= 1; ld >= cols; dtype SPX_DT_*; FP64 ops need SPX_DT_F64.
 *   lowp_ptr / lowp_ld: optional low-precision copy of the tile (NULL, 0).
 * Errors: SPX_ERR_INVALID_ARG, SPX_ERR_STATE (graph already executed). */
int spx_tile_register(spx_graph_t g, void* dev_ptr, int rows, int cols, int ld, int dtype,
                      void* lowp_ptr, int lowp_ld, unsigned* out_handle);

/* Register a low-precision matrix (BF16, or FP32 read as TF32) that holds the
 * low-precision copies of tiles (the lowp_ptr of spx_tile_register must
 * point inside it).  The library builds a TMA tensor map for it (128-row x
 * 128-byte boxes, 128-byte swizzle).  dev_ptr 16-byte aligned, ld * element
 * size a multiple of 16.  Registering the same base again returns the same
 * map.  Errors: SPX_ERR_INVALID_ARG, SPX_ERR_STATE, SPX_ERR_CUDA. */
int spx_lowp_register(spx_graph_t g, void* dev_ptr, int rows, int cols, int ld, int dtype,
                      unsigned* out_map);

/* Bytes of one split slot of an SPX_F64_OZAKI tile with pitch b: eight BF16
 * digit planes of b x b cut into 16-column chunks (plane s, row r, column k
 * at element ((s * (b / 16) + k / 16) * b + r) * 16 + k % 16), then b int32
 * row exponents, rounded up to 256 bytes.  0 for a b that spx_ozaki_register
 * rejects. */
long long spx_ozaki_slot_bytes(int b);

/* Register a store of nslots split slots (consecutive, spx_ozaki_slot_bytes(b)
 * bytes apart from dev_ptr, which must be 256-byte aligned) for
 * SPX_F64_OZAKI tasks: the lowp_ptr of a tile registered with
 * spx_tile_register must then be a slot's address, with lowp_ld = b and the
 * tile's rows, cols <= b.  b a multiple of 32, 32 <= b <= 512.  The library
 * builds two TMA tensor maps over the store (128- and 64-row boxes of one
 * 16-digit chunk of all eight planes, 32-byte swizzle).  Registering the same base
 * again returns the same map.  Errors: SPX_ERR_INVALID_ARG, SPX_ERR_STATE,
 * SPX_ERR_CUDA. */
int spx_ozaki_register(spx_graph_t g, void* dev_ptr, int nslots, int b, unsigned* out_map);

/* Insert one task (paper, section "Task insertion": one thread inserts tasks
 * with their accesses; the result equals running them in insertion order).
 *   op        SPX_OP_*; handles[nh] in the op's operand order; modes[nh] the
 *             access mode of each operand; 1 <= nh <= 16 (NOP/SPIN), fixed
 *             for the other ops; operand shapes must agree.
 *   priority  0 = normal, >0 = high (popped first; a hint, paper section
 *             "Task insertion" / "Scheduling"); >= 2 also marks the task as
 *             on the critical path: its POTRF, TRSM and FP64 SYRK / GEMM phases
 *             are cut into smaller parts (16-row / 32 x 32 units instead of 64),
 *             trading some per-part overhead for more SMs on the task.
 *   prec      SPX_F64, or SPX_TF32 / SPX_BF16 for TRSM, SYRK, GEMM_NT_SUB
 *             whose factor tiles have low-precision copies in a matrix
 *             registered with spx_lowp_register of the matching type;
 *             SPX_F64_OZAKI for TRSM, SYRK, GEMM_NT_SUB, TRTRI, TRSM_INV,
 *             POTRF_PANEL, GEMM_NN_ADD, SPLIT and SPLIT_T whose split
 *             operands have slots in a store registered with
 *             spx_ozaki_register.
 *   out_task  receives the task id (0, 1, 2, ... in insertion order); may be
 *             NULL.
 * Errors: SPX_ERR_INVALID_ARG, SPX_ERR_BAD_HANDLE, SPX_ERR_STATE. */
int spx_task_insert(spx_graph_t g, int op, const unsigned* handles, const int* modes, int nh,
                    int priority, int prec, unsigned* out_task);

/* Set a task's integer argument: for POTRF the global column offset of the
 * tile (info reports offset + local column, 1-based); for SPIN the spin time
 * in nanoseconds.  Errors: SPX_ERR_BAD_HANDLE, SPX_ERR_STATE. */
int spx_task_set_arg(spx_graph_t g, unsigned task, long long arg);

/* Set the scalar of an AXPY task (Y <- Y + alpha X; alpha 1 by default).
 * Errors: SPX_ERR_BAD_HANDLE, SPX_ERR_STATE, SPX_ERR_INVALID_ARG (not an
 * AXPY task, or alpha not finite or zero). */
int spx_task_set_scalar(spx_graph_t g, unsigned task, double alpha);

/* Criticality (the paper blames its Cholesky variance on scheduling without
 * it, section "Numerical applications"): replace every task's priority by
 * one computed from the longest paths of the DAG.  Each task weighs its
 * number of phases (its length in dependent steps); the top level t(u) is
 * the longest weighted path ending before u, the bottom level b(u) the
 * longest starting at u (u included), CP = max (t + b), slack(u) = CP -
 * t(u) - b(u).  Slack 0 (on a longest path): class 2 (critical-path queue,
 * finer parts); slack <= CP / 10: class 1; else 0.  Both levels come from the
 * access records in one forward and one backward pass over the tasks, with
 * per-handle group maxima (the STF groups give each task's predecessors and
 * successors), without the derived DAG.  Host only; the graph must be built
 * and not running.  Errors: SPX_ERR_INVALID_ARG, SPX_ERR_STATE. */
int spx_graph_assign_priorities(spx_graph_t g);

/* Derive the dependency DAG on the device (successor CSR sorted ascending,
 * de-duplicated, and in-degrees) without executing it.  Asynchronous on
 * stream.  Errors: SPX_ERR_STATE (no tasks), SPX_ERR_OOM, SPX_ERR_CUDA. */
int spx_graph_derive(spx_graph_t g, void* stream);

/* Derive (if not done) and launch the graph, asynchronously on stream.  The
 * graph is then running until spx_graph_wait returns.
 * Errors: SPX_ERR_STATE (running, or empty), SPX_ERR_OOM, SPX_ERR_CUDA. */
int spx_graph_execute(spx_graph_t g, void* stream);

/* Run several independently built graphs in one persistent launch (the
 * batched form of spx_graph_execute; the paper's runtime runs each task-graph
 * object on its own, section "Task graph description"; batching many small
 * graphs into one launch is this library's).
 *   gs[ng]   graphs that are built and not running (spx_graph_reset a
 *            finished one first), each with at least one task, all distinct.
 * The graphs' tiles, low-precision matrices and tasks are merged, members in
 * the order gs[0], gs[1], ..., tasks in their insertion order, into one
 * graph that gs[0] owns (kept for its next batch; freed with gs[0]); its DAG
 * is derived on the device and run by one persistent kernel with gs[0]'s
 * configuration (num_ctas, trace, no_split, watchdog; the members' own
 * executors are not used).  Graphs that share no tile address run as if
 * each ran alone, with bit-identical results for deterministic tile ops; a
 * tile address registered in several members orders their accesses as if
 * the members ran one after another.
 * Every member is then running.  spx_graph_wait on a member waits for the
 * launch and returns that member's own status: a POTRF that fails in one
 * member (SPX_NOT_SPD, info = its column) skips only that member's later
 * tasks, the other members finish normally; a run-wide error (watchdog,
 * queue) is returned for every member.  spx_graph_timing and spx_graph_stats
 * on a finished member report the whole launch; spx_graph_edges, tickets and
 * trace are not available for members.  After spx_graph_reset a member can
 * run alone or in another batch.
 * Errors: SPX_ERR_INVALID_ARG (NULL, ng < 1, a graph given twice, or tiles
 * of one address with different shapes), SPX_ERR_STATE (a graph running,
 * finished and not reset, or empty), SPX_ERR_OOM, SPX_ERR_CUDA. */
int spx_batch_execute(spx_graph_t* gs, int ng, void* stream);

/* Streaming (paper, section "Background" / "Task insertion": tasks are
 * inserted while the workers execute earlier ones).  spx_stream_begin
 * launches the persistent kernel on the tasks inserted so far (possibly none)
 * and keeps it running; spx_task_insert (on tiles registered before the
 * begin) may then be called while it runs, and spx_stream_flush hands the
 * tasks inserted since the last flush to the kernel (asynchronously: their
 * descriptors and predecessor lists are copied by the copy engine, then the
 * count the kernel polls is raised on the same stream); spx_stream_end flushes and lets the kernel finish and exit, after
 * which spx_graph_wait returns the run's status as for spx_graph_execute.
 *
 * Dependencies are derived on the host as each task is inserted, by the same
 * rule as the device derivation (see spx_graph_host_preds); the kernel
 * admits each published task by attaching it to its predecessors' successor
 * lists (64 slots per task; a predecessor whose list fills gets a relay: a
 * NOP task appended to the graph that depends on it and takes its later
 * successors) and runs it when they have finished.  Results equal running
 * the tasks in insertion order.
 *   max_tasks, max_tiles, max_records, max_preds: capacities for the whole
 *   stream (tasks including relays; tiles, all registered before the begin;
 *   access records; predecessor entries).
 *   The graph's configuration must be the persistent executor without CUDA
 *   graph replay or no_split; critical-path priorities are not assigned.
 *   The kernel family (FP64, tensor-core or split tasks) is fixed by the
 *   tasks inserted before the begin: a later task that needs another family
 *   is refused.
 *   The device watchdog (cfg.watchdog_ns) also bounds the host: the kernel
 *   leaves with SPX_ERR_TIMEOUT if no task finishes and none is published
 *   for that long before the end.
 * Errors (begin): SPX_ERR_INVALID_ARG (capacities below the tasks inserted
 * so far, configuration), SPX_ERR_STATE (not a graph being built), SPX_ERR_OOM,
 * SPX_ERR_CUDA.  spx_task_insert while streaming also returns
 * SPX_ERR_QUEUE_FULL when a capacity would be exceeded (the stream then
 * refuses further tasks; what was published still runs). */
int spx_stream_begin(spx_graph_t g, void* stream, int max_tasks, int max_tiles,
                     long long max_records, long long max_preds);
int spx_stream_flush(spx_graph_t g);
int spx_stream_end(spx_graph_t g);

/* Copy tile data from host memory to the device while streaming, ordered
 * before the next flush: the tasks flushed after this call read the copied
 * data (the copy runs on the stream's upload stream, ahead of the count the
 * kernel polls).  rows x width_bytes from host_src (row pitch spitch) to
 * dev_dst (row pitch dpitch), as cudaMemcpy2DAsync; host_src should be
 * pinned (a pageable source is staged before the call returns).  The data
 * must not be touched by a task published earlier.
 * Errors: SPX_ERR_INVALID_ARG, SPX_ERR_STATE (not streaming), SPX_ERR_CUDA. */
int spx_stream_copy_h2d(spx_graph_t g, void* dev_dst, size_t dpitch, const void* host_src,
                        size_t spitch, size_t width_bytes, size_t rows);

/* The predecessor lists of the inserted tasks as the host-side derivation of
 * a stream computes them (CSR by task: pred_ptr[ntasks + 1], pred[cap]); no
 * device work.  The edge set is the device derivation's (spx_graph_edges),
 * transposed.  total receives the number of entries; SPX_ERR_QUEUE_FULL if
 * above cap (pred then holds the first cap). */
int spx_graph_host_preds(spx_graph_t g, unsigned* pred_ptr, unsigned* pred, long long cap,
                         long long* total);

/* Wait for a running graph.  timeout_ns = 0 waits without a host limit (the
 * device watchdog still bounds the run).  info (may be NULL) receives the
 * LAPACK-style column of a failed POTRF, else 0.
 * Returns SPX_OK, SPX_NOT_SPD, SPX_ERR_TIMEOUT (device watchdog fired, or
 * host timeout: then the graph stays running and wait may be called again),
 * SPX_ERR_QUEUE_FULL, SPX_ERR_BAD_OP, SPX_ERR_CUDA, SPX_ERR_STATE. */
int spx_graph_wait(spx_graph_t g, unsigned long long timeout_ns, int* info);

/* Sizes: tasks, unique edges (valid after derive), accesses, tiles.  Any
 * output pointer may be NULL. */
int spx_graph_sizes(spx_graph_t g, long long* ntasks, long long* nedges, long long* naccesses,
                    long long* ntiles);

/* Copy the derived DAG to host arrays: row_ptr[ntasks+1], col[nedges],
 * indeg[ntasks] (any may be NULL).  Successors of task u are
 * col[row_ptr[u] .. row_ptr[u+1]) in ascending order.  Synchronises with the
 * graph's last stream.  Errors: SPX_ERR_STATE (not derived), SPX_ERR_CUDA. */
int spx_graph_edges(spx_graph_t g, unsigned* row_ptr, unsigned* col, unsigned* indeg);

/* Execution tickets of the last run: a global counter taken when a task's
 * first part starts (start[t]) and when its last part ends (end[t]).  For
 * every edge u->v, end[u] < start[v].  Errors: SPX_ERR_STATE. */
int spx_graph_tickets(spx_graph_t g, unsigned* start, unsigned* end);

/* Completion of tasks of a running (or streaming, or finished) graph on the
 * persistent executor: done[i] = 1 when task tasks[i] has finished (its
 * results are in memory and no later task of the graph writes them unless it
 * depends on it), else 0.  Reads a snapshot of the device's end tickets by
 * the copy engine while the kernel runs (microseconds; poll with a pause).
 * Errors: SPX_ERR_INVALID_ARG, SPX_ERR_BAD_HANDLE, SPX_ERR_STATE (not
 * launched, another executor, a batched member), SPX_ERR_CUDA. */
int spx_graph_tasks_done(spx_graph_t g, const unsigned* tasks, int count, int* done);

/* Trace of the last run with cfg.trace = 1 (paper, section "Visualization"):
 * 4 values per task: start ns, end ns (device %globaltimer), SM id of the
 * first part, number of parts.  Errors: SPX_ERR_STATE (tracing off). */
int spx_graph_trace(spx_graph_t g, unsigned long long* rec);

/* Op (SPX_OP_*) and scheduling class (0 normal, 1 high, 2 critical path) of
 * every task, in insertion order: ops[ntasks], priorities[ntasks] (either may
 * be NULL).  Host data only; any state.  Labels for traces (paper, section
 * "Visualization").  Errors: SPX_ERR_INVALID_ARG. */
int spx_graph_task_ops(spx_graph_t g, int* ops, int* priorities);

/* Counters of the last run: out[0] task parts executed, out[1] queue
 * high-water mark (entries), out[2] pops that found the queue empty,
 * out[3] CTAs used, out[4] busy cycles summed over CTAs, out[5] total
 * cycles summed over CTAs, out[6] queue capacity (entries per priority),
 * out[7] / out[8] entries pushed to the high (critical path and high) /
 * normal priority queues, out[9 + op] busy cycles of the parts of each op
 * (SPX_OP_*), summed over CTAs.  n = number of values wanted
 * (<= 9 + SPX_NUM_OPS). */
int spx_graph_stats(spx_graph_t g, long long* out, int n);

/* Device time of the last execution, from CUDA events recorded on the
 * execute stream: prep_ms = queue/state reset plus DAG derivation (or the
 * re-initialisation of a reset graph), run_ms = the executor (the persistent
 * kernel, or all per-task launches).  Either pointer may be NULL.
 * Errors: SPX_ERR_STATE (no finished execution). */
int spx_graph_timing(spx_graph_t g, float* prep_ms, float* run_ms);

/* Write the derived task graph in Graphviz dot format (paper, section
 * "Visualization", generateDot).  Errors: SPX_ERR_STATE, SPX_ERR_INVALID_ARG
 * (cannot open path). */
int spx_graph_write_dot(spx_graph_t g, const char* path);

/* Make an executed graph runnable again with the same DAG (no new
 * derivation).  The caller restores the tile contents.  With
 * cfg.cuda_graph = 1 the next execute replays one CUDA graph.
 * Errors: SPX_ERR_STATE. */
int spx_graph_reset(spx_graph_t g);

/* Drop all tiles and tasks but keep the allocations, so a new graph of a
 * similar size can be built without new device allocations. */
int spx_graph_clear(spx_graph_t g);

/* Free the graph.  Waits for a running graph first.  NULL is ignored. */
void spx_graph_destroy(spx_graph_t g);

/* Insert the whole tiled Cholesky of the paper's numerical applications
 * (section "Numerical applications": POTRF on diagonal tiles, TRSM, SYRK and
 * GEMM on the others), right-looking with k outer:
 *   for k: POTRF(k); TRSM(i,k) for i>k; SYRK(i,k) for i>k;
 *          GEMM(i,j,k) for j>k, i>j (j outer)
 * and, when dev_X != NULL, the block solve A Y = X (Y over X): forward
 * TRSM_L_FWD(k), GEMM_FWD(i,k) for k ascending, then backward
 * TRSM_LT_BWD(k), GEMM_BWD(i,k) for k descending.
 *   dev_A   n x n FP64 row-major (lda >= n); the lower triangle is replaced by
 *           L, the strict upper triangle is not touched.  Tiles are b x b
 *           (the last tile row/column is ragged when b does not divide n).
 *   dev_X   n x nrhs FP64 row-major (ldx >= nrhs) or NULL.
 *   lookahead  1: POTRF, TRSM, SYRK, the GEMMs of the next panel column and
 *           the diagonal solves get the high priority; 2: every task on
 *           the critical-path queue with the finer parts (the latency form
 *           for small problems, whose DAG is essentially one chain); 0: all
 *           tasks normal.
 *   prec    SPX_F64.
 *   out_ntasks  number of tasks inserted (may be NULL).
 * Errors: as spx_tile_register / spx_task_insert; tasks inserted before an
 * error stay in the graph. */
int spx_cholesky_insert(spx_graph_t g, double* dev_A, int n, int lda, int b, double* dev_X,
                        int nrhs, int ldx, int lookahead, int prec, long long* out_ntasks);

/* Mixed-precision form of spx_cholesky_insert: POTRF and the solves in FP64,
 * TRSM / SYRK / GEMM with prec = SPX_TF32 or SPX_BF16 (see the prec enum):
 * the trailing updates run on the tensor cores from low-precision copies of
 * the factor tiles kept in dev_Alo (n x n, ld ldlo; BF16 for SPX_BF16, FP32
 * for SPX_TF32; rows 16-byte aligned), which the TRSM tasks write.  b must be
 * a multiple of 64.  The resulting factor is accurate to the low precision;
 * pair it with FP64 iterative refinement (spx_residual_f64, spx_solve_insert). */
int spx_cholesky_insert_mixed(spx_graph_t g, double* dev_A, int n, int lda, int b, void* dev_Alo,
                              int ldlo, double* dev_X, int nrhs, int ldx, int lookahead, int prec,
                              long long* out_ntasks);

/* spx_cholesky_insert_mixed with the panel solves on the tensor cores: per
 * k, POTRF(k) in FP64, the critical panel tile TRSM(k+1, k) by FP64
 * substitution (it is on the critical path, and must not wait for the
 * inversion), TRTRI(k) writes V_k = L_kk^{-1} (FP64) into the square block at
 * row k*b of dev_V (n x b FP64 row-major, ldv >= b), and TRSM_INV(i, k) for
 * i >= k+2 forms A_ik V_k^T on the tensor cores from split TF32 operands
 * (about FP32 accuracy, see the prec enum) and writes the low-precision copy
 * of the result.  The TRSM tasks' b^3 flops per tile leave
 * the FP64 pipe, which they held for most of the mixed factorization's time
 * (the factor is only accurate to the low precision anyway).  On return dev_V
 * holds the inverses of all diagonal factor tiles, ready for the correction
 * solves of refinement (spx_solve_inv_insert, spx_solve_inv_f32_insert).
 * Solving with the diagonal inverses instead of substituting is a reading of
 * this library, not of the paper (whose TRSM task is a library call).
 * b a multiple of 64.  Errors: as spx_cholesky_insert_mixed, and
 * SPX_ERR_INVALID_ARG for a NULL dev_V or ldv < b. */
int spx_cholesky_insert_mixed_inv(spx_graph_t g, double* dev_A, int n, int lda, int b,
                                  void* dev_Alo, int ldlo, double* dev_V, int ldv, double* dev_X,
                                  int nrhs, int ldx, int lookahead, int prec,
                                  long long* out_ntasks);

/* spx_cholesky_insert with the trailing updates in FP64 emulated on the
 * tensor cores (prec SPX_F64_OZAKI, see the prec enum): POTRF and the solves
 * in FP64; TRSM solves in FP64 and splits its result into the slot of its
 * tile; SYRK and GEMM_NT_SUB run on the tensor cores from the slots.
 *   dev_S   the split store: the tile (i, k), i > k, uses slot
 *           i (i - 1) / 2 + k, i.e. T (T - 1) / 2 slots for T = ceil(n / b)
 *           (T more with dev_V, see below); S_bytes its size, at least that
 *           many times spx_ozaki_slot_bytes(b); 256-byte aligned.  The
 *           caller owns it and keeps it alive until the graph is waited for.
 *   dev_V   NULL: every panel tile by FP64 substitution.  Else inverse
 *           panels: per k, the critical panel tile (k+1, k) by FP64
 *           substitution; TRTRI writes V_k = L_kk^{-1} (FP64, block
 *           recursive) into the square block at row k*b of dev_V (n x b,
 *           ldv >= b) and splits it into slot T (T - 1) / 2 + k; TRSM_INV
 *           with the split prec then forms A_ik V_k^T for i >= k+2 as a split
 *           product (A_ik split, product stored, result split): the panel
 *           solves' b^3 flops per tile leave the FP64 pipe.  Substitution and
 *           the inverse agree to rounding for well-conditioned diagonal tiles
 *           (the error of the inverse grows with kappa(L_kk)); this is a
 *           reading of this library, not of the paper.
 *   fuse_panel  1: POTRF(k) and the solve of the critical panel tile
 *           (k+1, k) run as one SPX_OP_POTRF_PANEL task (the same arithmetic;
 *           the critical path crosses fewer phase and task boundaries); 0:
 *           separate POTRF and TRSM tasks.
 *   b       a multiple of 32, 32 <= b <= 512.
 * Other arguments as spx_cholesky_insert.  Errors: as spx_cholesky_insert,
 * and SPX_ERR_INVALID_ARG for b, the store, or ldv < b. */
int spx_cholesky_insert_ozaki(spx_graph_t g, double* dev_A, int n, int lda, int b, void* dev_S,
                              long long S_bytes, double* dev_V, int ldv, int fuse_panel,
                              double* dev_X, int nrhs, int ldx, int lookahead,
                              long long* out_ntasks);

/* End to end from host memory: the split-FP64 Cholesky of
 * spx_cholesky_insert_ozaki (inverse panels, look-ahead marks, no solve) of
 * the matrix in host_A (n x n FP64 row-major, ld_host; pinned memory for
 * asynchronous copies; the lower triangle is read), its factor written into
 * the lower triangle of host_L (same layout; the strict upper part of the
 * diagonal blocks receives dev_A's, the rest of the upper triangle is not
 * written).  The column blocks of the lower triangle are copied into dev_A
 * (n x n, lda) while the persistent kernel runs (streaming insertion: block
 * column j's first-step tasks are published after its copy, block 0 is
 * copied before the launch), then the factor's column blocks are copied
 * back after the run.  The same tasks and per-tile order as
 * spx_cholesky_insert_ozaki: the factor is bit-identical.  g: a graph being
 * built with no tasks (persistent executor); dev_S, S_bytes, dev_V, ldv as
 * in spx_cholesky_insert_ozaki (dev_V required); stream: the launch stream,
 * synchronised before the return.  Returns SPX_OK or SPX_NOT_SPD (info: the
 * failed column, 1-based) like spx_graph_wait, or an error as
 * spx_stream_begin / spx_task_insert / spx_graph_wait.  After the return
 * the graph is finished (spx_graph_reset / spx_graph_clear to reuse). */
int spx_cholesky_host_ozaki(spx_graph_t g, const double* host_A, double* host_L, int n,
                            int ld_host, int b, double* dev_A, int lda, void* dev_S,
                            long long S_bytes, double* dev_V, int ldv, void* stream, int* info);

/* Insert only the block solve tasks L L^T Y = X (Y over X) for a factor L
 * already in dev_L (lower triangle, tiles b x b).  Used for the correction
 * solves of iterative refinement; re-run with spx_graph_reset. */
int spx_solve_insert(spx_graph_t g, double* dev_L, int n, int ld, int b, double* dev_X, int nrhs,
                     int ldx, long long* out_ntasks);

/* Insert one TRTRI task per diagonal tile of the factor in dev_L (n x n,
 * lower, tiles b x b): V_k <- L_kk^{-1} into the square b_k x b_k block at
 * row k*b of dev_V (n x b FP64 row-major, ld ldv >= b; b_k = b, or the
 * ragged remainder for the last tile).  The block solve y_k = L_kk^{-1} b_k
 * can then apply each inverse as a product (spx_solve_inv_insert).
 * Errors: as spx_tile_register / spx_task_insert. */
int spx_trtri_insert(spx_graph_t g, double* dev_L, int n, int ldl, int b, double* dev_V, int ldv,
                     long long* out_ntasks);

/* Insert the block solve L L^T x = r with the diagonal inverses of
 * spx_trtri_insert applied as products: forward, for k ascending, y_k =
 * V_k (r_k - sum_{j<k} L_kj y_j); backward, for k descending, x_k = V_k^T
 * (y_k - sum_{i>k} L_ik^T x_i).  dev_R (n x nrhs, ldx) holds r on entry and
 * x on exit; dev_D (same shape) receives y.  One TRMM per block step
 * replaces the 2 nb - 1 dependent phases of a substitution, so the chain of
 * the solve is shorter; the result equals the substitution's up to rounding
 * (the products reassociate it).  Used for the correction solves of
 * iterative refinement; re-run with spx_graph_reset.
 * Errors: as spx_tile_register / spx_task_insert. */
int spx_solve_inv_insert(spx_graph_t g, double* dev_L, int n, int ldl, int b, double* dev_V,
                         int ldv, double* dev_R, double* dev_D, int nrhs, int ldx,
                         long long* out_ntasks);

/* The correction step of mixed-precision refinement with the solve in FP32:
 * COPY tasks round the FP64 residual dev_R (n x nrhs, ldx) into dev_R32, the
 * block solve of spx_solve_inv_insert runs on FP32 copies of the factor
 * (dev_L32: n x n row-major FP32, ld ldl, strictly lower tiles read) and of
 * the diagonal inverses (dev_V32: n x b FP32, ld ldv), with dev_D32 as its
 * forward result, and AXPY tasks add the correction to dev_X (FP64, ldx):
 * x <- x + (L L^T)^{-1} r.  The factor of a TF32 / BF16 Cholesky is only
 * accurate to that precision, so solving for the correction in FP32 does
 * not slow the refinement, and it runs on the FP32 pipe instead of FP64.
 * dev_R32 and dev_D32 are n x nrhs FP32 with ld ldx, distinct buffers;
 * 1 <= nrhs <= 16.  The copies are the caller's (FP64 -> FP32 of L and V,
 * e.g. with one COPY task each).  No counterpart in the paper (the workload
 * definition's refinement).
 * Errors: SPX_ERR_INVALID_ARG for null or aliased pointers, bad sizes or
 * nrhs > 16; otherwise as spx_tile_register / spx_task_insert. */
int spx_solve_inv_f32_insert(spx_graph_t g, const float* dev_L32, int n, int ldl, int b,
                             const float* dev_V32, int ldv, const double* dev_R, float* dev_R32,
                             float* dev_D32, double* dev_X, int nrhs, int ldx,
                             long long* out_ntasks);

/* Scheduler-overhead pattern of the paper's engine benchmark (section
 * "Results" of the overhead study): `chains` independent chains of `ntasks`
 * tasks; every task of chain c accesses the same `deps` data objects of that
 * chain (1 <= deps <= 16), all with SPX_WRITE, or all with
 * SPX_COMMUTATIVE_WRITE when `commutative` (then the tasks of a chain run in
 * any order, one at a time, under the objects' locks); each task busy-waits
 * spin_ns nanoseconds (SPX_OP_SPIN; SPX_OP_NOP when spin_ns = 0).  Tasks are
 * inserted round-robin over the chains.  Execution time ~ ntasks (spin + O),
 * O the per-task overhead of the executor.  The data objects are addresses
 * that are never dereferenced.
 * Errors: SPX_ERR_INVALID_ARG; as spx_tile_register / spx_task_insert. */
int spx_overhead_insert(spx_graph_t g, int chains, int ntasks, int deps, int commutative,
                        long long spin_ns, long long* out_ntasks);

/* Insert `sweeps` FP64 iterative-refinement sweeps as tasks (so that they run
 * inside the same graph, e.g. in the server): each sweep is
 *   R_i <- B_i (COPY);  R_i <- R_i - A0_ij X_j for all i, j (GEMM_FWD);
 *   L L^T D = R by the block solves (D over R);  X_i <- X_i + R_i (AXPY).
 * A0: n x n original matrix in full (lda); L: the factor (lower triangle of
 * dev_L, ldl); B, X, R: n x nrhs (ldx).  X holds the current solution. */
int spx_refine_insert(spx_graph_t g, double* dev_A0, int n, int lda, double* dev_L, int ldl, int b,
                      double* dev_B, double* dev_X, double* dev_R, int nrhs, int ldx, int sweeps,
                      long long* out_ntasks);

/* spx_refine_insert with the correction solves of spx_solve_inv_insert: one
 * TRTRI task per diagonal factor tile first (V_k <- L_kk^{-1} into dev_V,
 * n x b, ldv >= b), then each sweep applies the inverses as products, with
 * dev_D (n x nrhs, ldx) as the forward sweep's output.  Shorter chains per
 * sweep than the substitution form; same result up to rounding. */
int spx_refine_inv_insert(spx_graph_t g, double* dev_A0, int n, int lda, double* dev_L, int ldl,
                          int b, double* dev_V, int ldv, double* dev_B, double* dev_X,
                          double* dev_R, double* dev_D, int nrhs, int ldx, int sweeps,
                          long long* out_ntasks);

/* Insert the tiled GEMM C += A B of the paper's numerical applications: one
 * GEMM_NN_ADD task per (i, j, k), i and j outer, k inner, each with a WRITE
 * (commutative = 0), a COMMUTATIVE_WRITE (1: the tasks of a block run one at
 * a time in any order) or an ATOMIC_WRITE (2: the tasks of a block run at the
 * same time and add into it atomically) on the block C_ij.  A, B, C are
 * n x n FP64 row-major with leading dimension ld; tiles b x b.
 * Errors: SPX_ERR_INVALID_ARG; as spx_tile_register / spx_task_insert. */
int spx_gemm_insert(spx_graph_t g, double* dev_A, double* dev_B, double* dev_C, int n, int ld,
                    int b, int commutative, long long* out_ntasks);

/* spx_gemm_insert with the products in FP64 emulated on the tensor cores
 * (prec SPX_F64_OZAKI): first one SPLIT task per tile A_ik and one SPLIT_T
 * task per tile B_kj (row-major order of each matrix), then the GEMM_NN_ADD
 * tasks of spx_gemm_insert with the split prec, each reading the two slots
 * and adding its product into C_ij with one rounding per entry.
 *   dev_S   the split store: A_ik uses slot i T + k, B_kj slot T^2 + k T + j
 *           (2 T^2 slots, T = ceil(n / b)); S_bytes its size, at least that
 *           many times spx_ozaki_slot_bytes(b); 256-byte aligned; owned by
 *           the caller until the graph is waited for.
 *   commutative  0 (WRITE) or 1 (COMMUTATIVE_WRITE); the split product is
 *           not an atomic update, so 2 is SPX_ERR_INVALID_ARG.
 *   b       a multiple of 32, 32 <= b <= 512.
 * Error of one product entry: at most n_k 9.05 2^-56 2^(e_r + f_c) before its
 * rounding (n_k = the K extent, e_r and f_c the exponents of row r of A_ik
 * and column c of B_kj), FP64's level.
 * Errors: SPX_ERR_INVALID_ARG; as spx_ozaki_register / spx_tile_register /
 * spx_task_insert. */
int spx_gemm_insert_ozaki(spx_graph_t g, double* dev_A, double* dev_B, double* dev_C, int n,
                          int ld, int b, int commutative, void* dev_S, long long S_bytes,
                          long long* out_ntasks);

/* Insert the AXPY of the paper's numerical applications (section "Numerical
 * applications": a vector split into pieces, one independent task per piece,
 * single precision): y <- y + alpha x over n FP32 values (dev_x, dev_y
 * distinct device arrays), in pieces of `piece` values (the last one
 * ragged), one AXPY task per piece with x_p READ and y_p WRITE.  A piece is
 * registered as a (len / 1024) x 1024 tile when 1024 divides its length,
 * else as one row.  Each value is computed as fl(fl(alpha x) + y) (one
 * rounding when alpha = 1).
 * Errors: SPX_ERR_INVALID_ARG; as spx_tile_register / spx_task_insert. */
int spx_axpy_insert(spx_graph_t g, float* dev_x, float* dev_y, long long n, long long piece,
                    double alpha, long long* out_ntasks);

/* Insert the particle-interaction test case of the paper's numerical
 * applications (direct Coulomb summation in FP64; dependencies on whole
 * groups): ngroups groups, group i an sizes[i] x 8 FP64 tile at
 * dev_groups[i] (ld 8; x, y, z, q, phi, E, see SPX_OP_NBODY_SELF), tasks in
 * the order NBODY_SELF(i), then NBODY_PAIR(i, j) for j > i, for i = 0, 1,
 * ...; each task writes its groups (SPX_WRITE, or SPX_COMMUTATIVE_WRITE when
 * commutative: a group's accumulations may then run in any order).  phi and
 * E accumulate into the tiles (zero them first for the plain sums).
 * Errors: SPX_ERR_INVALID_ARG; as spx_tile_register / spx_task_insert. */
int spx_nbody_insert(spx_graph_t g, int ngroups, double* const* dev_groups, const int* sizes,
                     int commutative, long long* out_ntasks);

/* Largest inputs of spx_graph_derive_noalloc (its fixed scratch is sized
 * for these: about 5.3 MB of device memory per GPU). */
#define SPX_NOALLOC_MAX_RECORDS 262144
#define SPX_NOALLOC_MAX_HANDLES 65536

/* Dependency derivation that allocates nothing.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (a host callback, a runtime that owns every device byte through
 * its own pool, a server that must not touch the allocator while it serves)
 * and therefore cannot use a graph object, whose execute call allocates.
 * It computes the same successor CSR and in-degrees as spx_graph_derive, from
 * access records the caller already holds in device memory, using a fixed
 * scratch array inside the library instead of allocated scratch.
 *   dev_task_rec   [ntasks+1] first record of each task; task_rec[0] = 0,
 *                  task_rec[ntasks] = nrec, 1..16 records per task.
 *   dev_rec_handle [nrec] handle of each record (< nhandles); a task names a
 *                  handle at most once (merge repeated accesses first).
 *   dev_rec_seq    [nrec] position of the record on its handle's list: the
 *                  records of handle h, in task order, have 0, 1, 2, ...
 *   dev_rec_mode   [nrec] SPX_READ / SPX_WRITE / SPX_COMMUTATIVE_WRITE /
 *                  SPX_ATOMIC_WRITE / SPX_MAYBE_WRITE.
 *   dev_row_ptr    [ntasks+1] out; dev_col [col_cap] out; dev_indeg [ntasks]
 *                  out; dev_status [1] out (device int).
 * Asynchronous on stream.  Host-side errors (returned): SPX_ERR_INVALID_ARG
 * for NULL pointers, bad counts, or nrec > SPX_NOALLOC_MAX_RECORDS or
 * nhandles > SPX_NOALLOC_MAX_HANDLES; SPX_ERR_CUDA if the set-up or the launch
 * fails.  Device-side (in *dev_status once the stream reaches it): 0, or
 * SPX_ERR_INVALID_ARG for malformed records, or for col_cap smaller than the
 * number of edges E.  In the last case dev_col and dev_indeg are not written
 * and dev_row_ptr[ntasks] holds E, or 0xFFFFFFFF when E does not fit 32 bits
 * (E is summed in 64 bits: a valid list can have more than 2^32 edges, e.g.
 * 65536 READs followed by 65536 COMMUTATIVE_WRITEs on one handle); the other
 * dev_row_ptr entries are then unspecified.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the life
 * of the process; make that first call before any stream capture, and do not
 * call this function on a device after cudaDeviceReset (the kept address
 * belongs to the destroyed context).  Every call shares the scratch array:
 * calls that overlap on the GPU (other streams, other threads) race and give
 * wrong results; calls in sequence on one stream are independent. */
int spx_graph_derive_noalloc(const unsigned* dev_task_rec, const unsigned* dev_rec_handle,
                             const unsigned* dev_rec_seq, const unsigned char* dev_rec_mode,
                             int ntasks, int nhandles, long long nrec, unsigned* dev_row_ptr,
                             unsigned* dev_col, long long col_cap, unsigned* dev_indeg,
                             int* dev_status, void* stream);

/* Low-precision tile update on the tensor cores, stand-alone: the building
 * block of the mixed-precision SYRK / GEMM tasks (the trailing updates of the
 * paper's tiled Cholesky run in BF16 or TF32 with FP32 accumulation while the
 * trailing matrix stays FP64):
 *     C (m x n, FP64, ldc) -= A (m x K) * B (n x K)^T
 * A and B row-major low precision (prec SPX_BF16: bfloat16; SPX_TF32: FP32
 * storage whose low 13 mantissa bits the tensor core ignores), leading
 * dimensions lda, ldb in elements (rows 16-byte aligned).  tcgen05.mma with
 * TMEM accumulators, operands by TMA.  Asynchronous on stream; *dev_err (a
 * device int the caller zeroes) becomes 1 if a device wait timed out.
 * Errors: SPX_ERR_INVALID_ARG, SPX_ERR_CUDA. */
int spx_tc_gemm_nt(double* dev_C, int ldc, int m, int n, const void* dev_A, int lda,
                   const void* dev_B, int ldb, int K, int prec, int* dev_err, void* stream);

/* Insert `count` independent Cholesky solves into one graph (the batched
 * form of spx_cholesky_insert: problem i uses dev_A[i], n[i], lda[i], b[i],
 * dev_X[i] (may be NULL), nrhs[i], ldx[i]).  The problems share no tile, so
 * their DAGs are disjoint and one persistent launch runs all of them.
 * Host arrays of length count.  Errors as spx_cholesky_insert. */
int spx_cholesky_insert_batch(spx_graph_t g, int count, double* const* dev_A, const int* n,
                              const int* lda, const int* b, double* const* dev_X, const int* nrhs,
                              const int* ldx, int lookahead, int prec, long long* out_ntasks);

/* FP64 residual of iterative refinement: R = B - A X (A n x n, X, B, R
 * n x nrhs, all FP64 row-major with the given leading dimensions, R may not
 * alias X or B), 1 <= nrhs <= 16.  dev_norms [3*nrhs] receives max|r_j| at
 * [j], max|x_j| at [nrhs+j], max|b_j| at [2 nrhs+j], from which the
 * normwise backward error eta_j = max|r_j| / (||A||_inf max|x_j| + max|b_j|)
 * follows (Rigal-Gaches).  Asynchronous on stream.
 * Errors: SPX_ERR_INVALID_ARG, SPX_ERR_CUDA. */
int spx_residual_f64(const double* dev_A, int n, int lda, const double* dev_X, int ldx,
                     const double* dev_B, int ldb, double* dev_R, int ldr, int nrhs,
                     double* dev_norms, void* stream);

/* Residual and normwise backward error of iterative refinement, both on the
 * device: R = B - A X as in spx_residual_f64 (same arguments, norms in
 * dev_norms [3*nrhs]), then dev_eta[j] = max|r_j| / (||A||_inf max|x_j| +
 * max|b_j|) for j < nrhs (Rigal-Gaches normwise backward error, the
 * stopping test of the refinement) and dev_eta[nrhs] = max_j dev_eta[j].
 * dev_anorm [1] holds ||A||_inf (spx_norm_inf_f64).
 *   compensated = 0: plain FP64 FMA sums (the fast residual; its rounding
 *                    error is of the order gamma_n (|A||x| + |b|), as large as
 *                    eta itself once the refinement has converged).
 *   compensated = 1: every row summed with Dot2 (Ogita-Rump-Oishi 2005,
 *                    TwoProduct + TwoSum with separately summed errors):
 *                    R is as accurate as a residual computed in twice the
 *                    working precision and rounded, so eta bounds the
 *                    backward error of X to a relative O(u); about ten FP64
 *                    operations per term instead of one.
 * No counterpart in the paper (the workload definition's refinement).
 * Asynchronous on stream.  Errors: SPX_ERR_INVALID_ARG (as spx_residual_f64,
 * or NULL dev_anorm / dev_eta, or compensated not 0 / 1), SPX_ERR_CUDA. */
int spx_residual_eta_f64(const double* dev_A, int n, int lda, const double* dev_X, int ldx,
                         const double* dev_B, int ldb, double* dev_R, int ldr, int nrhs,
                         const double* dev_anorm, double* dev_norms, double* dev_eta,
                         int compensated, void* stream);

/* GMRES-based iterative refinement (Carson and Higham 2017, 2018; the
 * paper's refinement is the workload definition's, its GMRES form this
 * library's): solve A X = B (A n x n FP64, lda; B, X n x nrhs FP64 row-major,
 * ld = nrhs, 1 <= nrhs <= 16; X holds the first solution on entry) by
 * refinement steps whose correction equation A d = r is solved by GMRES on
 * M^{-1} A d = M^{-1} r, M = L L^T the low-precision factor.  precond is a
 * solve graph the caller built over dev_R (n x nrhs FP64, ld = nrhs): one
 * execution must leave M^{-1} R in dev_R (e.g. spx_solve_inv_insert or
 * spx_solve_insert on the factor); the driver resets and runs it as needed.
 * Each step: the residual and its normwise backward error on the device
 * (spx_residual_eta_f64 logic: plain residuals until eta <= tol or eta stops
 * falling, then compensated ones, so the final eta is certified), then up to
 * max_inner GMRES iterations (FP64; CGS2 orthogonalisation; Givens
 * rotations; all right-hand sides in lockstep) until the largest relative
 * GMRES residual is <= inner_tol, then x += d.  dev_work: device workspace of
 * spx_gmres_ir_workspace(n, nrhs, max_inner) bytes (the call allocates
 * nothing).  Synchronous on stream (it reads device scalars to decide).
 * Returns SPX_OK with out filled (converged or not: non-convergence is
 * reported, never hidden), or an error of the precond graph, or
 * SPX_ERR_INVALID_ARG / SPX_ERR_CUDA. */
typedef struct {
  int max_outer;     /* refinement steps (0 = 20)                         */
  int max_inner;     /* GMRES iterations per step, <= 64 (0 = 30)         */
  double inner_tol;  /* relative GMRES residual (0 = 1e-10)               */
  double tol;        /* target normwise backward error (0 = 1e-14)        */
} spx_gmres_config_t;

typedef struct {
  int converged;     /* 1 when the certified eta <= tol                   */
  int outer;         /* refinement steps taken                            */
  int inner;         /* GMRES iterations over all steps                   */
  int pad_;
  double eta;        /* last (compensated when converged) max eta         */
} spx_gmres_result_t;

long long spx_gmres_ir_workspace(int n, int nrhs, int max_inner);

int spx_gmres_ir(const double* dev_A, int n, int lda, const double* dev_B, double* dev_X, int nrhs,
                 spx_graph_t precond, double* dev_R, void* dev_work, long long work_bytes,
                 const spx_gmres_config_t* cfg, spx_gmres_result_t* out, void* stream);

/* ||A||_inf (max row sum of |a_ij|) of an n x n FP64 matrix into dev_out[0]. */
int spx_norm_inf_f64(const double* dev_A, int n, int lda, double* dev_out, void* stream);

/* Y += alpha X over count contiguous FP64 values (the refinement update). */
int spx_axpy_f64(double* dev_Y, const double* dev_X, long long count, double alpha, void* stream);

/* ---- Continuous-batching server ------------------------------------------
 * One resident persistent kernel runs the tasks of every live request; new
 * requests are admitted while it runs (the serving form of the executor: the
 * paper's runtime keeps accepting tasks while workers compute, section
 * "Background" / "Task insertion").  A request is a graph built with the
 * calls above and not executed; the server copies it (the graph may be
 * cleared or destroyed after submit returns, the tile memory must live until
 * the request is done).  Requests may not use COMMUTATIVE_WRITE; low-precision
 * tasks need tensor_cores >= 1, split-FP64 tasks (SPX_F64_OZAKI) need
 * tensor_cores = 2. */
typedef struct spx_server* spx_server_t;

typedef struct {
  long long max_tasks;       /* pool sizes shared by all live requests       */
  long long max_tiles;
  long long max_records;
  long long max_edges;
  long long max_maps;
  long long queue_capacity;  /* ring entries per priority                    */
  int num_ctas;              /* resident CTAs; 0 = resident maximum          */
  int tensor_cores;          /* 0 = FP64 tile ops only (two CTAs per SM);
                                1 = with the TF32/BF16 tensor-core ops;
                                2 = one CTA per SM owning all of TMEM: also
                                the split-FP64 products (SPX_F64_OZAKI)     */
  unsigned long long watchdog_ns; /* live work without progress -> error     */
  unsigned long long idle_ns;     /* resident kernel exits when idle this long
                                     (relaunched by the next submit/poll)   */
} spx_server_config_t;

void spx_server_config_default(spx_server_config_t* cfg);

/* Allocate the pools (one device arena) and the host-mapped control block.
 * Errors: SPX_ERR_INVALID_ARG, SPX_ERR_OOM, SPX_ERR_CUDA. */
int spx_server_create(spx_server_t* out, const spx_server_config_t* cfg);

/* Copy graph g into the pools and publish it; the resident kernel derives
 * its DAG on the device and interleaves its tasks with the other requests'.
 * Launches the resident kernel if it is not running.  *out_request receives
 * the request id.  SPX_ERR_OOM: no room now (pools, request slots or queue
 * entries) - poll finished requests and retry (admission).  Errors also:
 * SPX_ERR_INVALID_ARG, SPX_ERR_STATE, SPX_ERR_CUDA, or the server's failure
 * status (SPX_ERR_TIMEOUT, SPX_ERR_QUEUE_FULL) if its kernel died. */
int spx_server_submit(spx_server_t s, spx_graph_t g, unsigned long long* out_request);

/* 1 when the request finished (status: SPX_OK or SPX_NOT_SPD with info, its
 * pool ranges are freed and the id becomes invalid), 0 while it runs,
 * negative on error (SPX_ERR_BAD_HANDLE for an unknown id). */
int spx_server_poll(spx_server_t s, unsigned long long request, int* status, int* info);

/* Let the resident kernel finish the live requests and exit; returns its
 * status.  The server can be used again afterwards. */
int spx_server_stop(spx_server_t s);

/* Counters (after stop): out[0] parts run, out[1] tasks finished, out[2]
 * requests claimed, out[3] requests live, out[4] busy cycles, out[5] total
 * cycles.  n <= 6.  SPX_ERR_STATE while the kernel runs. */
int spx_server_stats(spx_server_t s, long long* out, int n);

void spx_server_destroy(spx_server_t s);

/* Strided 2-D copy by the copy engines (cudaMemcpy2DAsync, any direction):
 * rows x width_bytes from src (row pitch spitch) to dst (dpitch).  Used to
 * stage request inputs while a resident server kernel holds every SM. */
int spx_copy2d(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width_bytes,
               size_t rows, void* stream);

/* Static description of a status code. */
const char* spx_strerror(int code);

/* Library ABI version (incremented on incompatible changes). */
int spx_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPX_H_ */
