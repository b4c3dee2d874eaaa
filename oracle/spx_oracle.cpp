// CPU ORACLE — test infrastructure, not part of the product.
//
// Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
// may load this library.  It shares no code with the CUDA path: every
// function below is written from the Specx paper (arXiv 2308.15964) and from
// the textbook definitions it relies on, plain and slow on purpose.
//
// What it computes, and the passage each part follows:
//   * spxo_derive      - STF dependency derivation.  Section "Internal
//                        implementation": one data handle per address kept in
//                        an unordered hash map, each handle holding the
//                        ordered list of the tasks that use it; section "Task
//                        insertion" for the access modes SpRead / SpWrite /
//                        SpCommutativeWrite.  Output: explicit successor CSR.
//   * spxo_execute     - sequential semantics of the STF model (section
//                        "Background" / "Task insertion": the result equals
//                        running the tasks one after the other in insertion
//                        order).  Runs the tile tasks of the tiled Cholesky of
//                        section "Numerical applications" (POTRF, TRSM, SYRK,
//                        GEMM) plus GEMM-DAG and block-solve tasks, each as a
//                        plain FP64 loop nest, no blocking, no BLAS.
//   * spxo_potrf / spxo_trsv_* - unblocked Cholesky (Cholesky-Crout, column
//                        by column) and forward/back substitution; used both
//                        as the POTRF tile op and as the untiled reference.
//   * spxo_trtri       - inverse of a lower-triangular tile by forward
//                        substitution on the identity (the block solve can
//                        apply L_kk^{-1} as a product: y_k = L_kk^{-1} b_k).
//   * metrics          - factor backward error ||A-LL^T||_F/||A||_F,
//                        normwise backward error of a solve (Rigal-Gaches),
//                        a Freivalds-style probe; residual sums use the
//                        compensated dot product of Ogita, Rump and Oishi
//                        (2005) so the metric itself is accurate to ~u.
//
// Parity pins for every function live in tests/test_oracle_*.py.
//
// Build: g++ -O2 -ffp-contract=off -fno-fast-math -shared -fPIC (see
// oracle/oracle.py).  Floating point is IEEE binary64 round-to-nearest with no
// contraction, so each sum is evaluated left to right exactly as written.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <unordered_map>
#include <utility>
#include <vector>
#include <chrono>
#include <thread>

extern "C" {

// Access modes (section "Task insertion").
// Access modes (section "Task insertion"): SpRead, SpWrite,
// SpCommutativeWrite, SpAtomicWrite (handled like a read by the runtime: a run
// of them is one group; the task protects its own writes) and SpMaybeWrite
// (a possible write; without speculation it orders exactly like a write).
enum { O_READ = 0, O_WRITE = 1, O_COMMUTE = 2, O_ATOMIC = 3, O_MAYBE = 4 };

// Tile operations of the tiled Cholesky (section "Numerical applications")
// and of the block solve / tiled GEMM workloads.
enum {
  O_POTRF = 0,        // A_kk = L_kk L_kk^T, lower, in place
  O_TRSM = 1,         // A_ik <- A_ik L_kk^{-T}
  O_SYRK = 2,         // A_ii <- A_ii - L_ik L_ik^T (lower triangle)
  O_GEMM_NT_SUB = 3,  // A_ij <- A_ij - L_ik L_jk^T
  O_GEMM_NN_ADD = 4,  // C_ij <- C_ij + A_ik B_kj
  O_TRSM_L_FWD = 5,   // X_k <- L_kk^{-1} X_k
  O_GEMM_FWD = 6,     // X_i <- X_i - L_ik X_k
  O_TRSM_LT_BWD = 7,  // X_k <- L_kk^{-T} X_k
  O_GEMM_BWD = 8,     // X_i <- X_i - L_ki^T X_k
  O_NOP = 9,
  O_SPIN = 10,
  O_COPY = 11,        // Y <- X
  O_AXPY = 12,        // Y <- Y + X
  O_TRMM = 13,        // Y <- T X (arg 0) or T^T X (arg 1), T lower triangular
  O_TRTRI = 14,       // V <- L^{-1}, L lower triangular
  O_TRSM_INV = 15,    // A_ik <- A_ik V^T, V = L_kk^{-1} (the TRSM by the inverse)
  O_NBODY_SELF = 16,  // Coulomb interactions inside one particle group
  O_NBODY_PAIR = 17,  // interactions between two groups, both updated
  O_POTRF_PANEL = 18  // POTRF of A_kk, then A_ik <- A_ik L_kk^{-T}
};

// ---------------------------------------------------------------------------
// DAG derivation
// ---------------------------------------------------------------------------

// One group on a handle's dependency list: a run of READs, a run of
// COMMUTATIVE_WRITEs inserted one after the other, a run of ATOMIC_WRITEs, or
// a single WRITE or MAYBE_WRITE.
struct Group {
  int mode;
  std::vector<uint32_t> tasks;
};

// Merge two modes of the same task on the same handle.  The paper is silent;
// the reading used here: the same mode twice stays that mode (READ+READ =
// READ, COMM+COMM = COMM, ATOMIC+ATOMIC = ATOMIC, MAYBE+MAYBE = MAYBE), any
// two different modes give WRITE.
static int merge_mode(int a, int b) {
  if (a == b) return a;
  return O_WRITE;
}

// Derive the successor CSR of the task graph.
//   accesses are given in insertion order: acc_task[] is non-decreasing.
//   row_ptr[ntasks+1], indeg[ntasks] are written; col[] is written only when
//   the edge count fits col_cap.  Returns the number of unique edges, or -1
//   on malformed input.
long long spxo_derive(int ntasks, long long nacc, const uint32_t* acc_task,
                      const uint64_t* acc_key, const int* acc_mode,
                      uint32_t* row_ptr, uint32_t* indeg, uint32_t* col,
                      long long col_cap) {
  std::unordered_map<uint64_t, std::vector<Group>> handles;
  std::vector<std::pair<uint32_t, uint32_t>> edges;

  long long a = 0;
  while (a < nacc) {
    const uint32_t t = acc_task[a];
    if ((int)t >= ntasks) return -1;
    if (a > 0 && acc_task[a - 1] > t) return -1;
    // Collect this task's accesses, merging repeated keys.
    std::vector<std::pair<uint64_t, int>> mine;
    while (a < nacc && acc_task[a] == t) {
      const int m = acc_mode[a];
      if (m < O_READ || m > O_MAYBE) return -1;
      bool found = false;
      for (auto& km : mine) {
        if (km.first == acc_key[a]) {
          km.second = merge_mode(km.second, m);
          found = true;
        }
      }
      if (!found) mine.push_back({acc_key[a], m});
      ++a;
    }
    // Append the task to each handle's list.
    for (auto& km : mine) {
      std::vector<Group>& list = handles[km.first];
      const int m = km.second;
      const bool joins = !list.empty() && list.back().mode == m &&
                         (m == O_READ || m == O_COMMUTE || m == O_ATOMIC);
      if (joins) {
        // Same run as the last group: depends on the group before it.
        if (list.size() >= 2) {
          for (uint32_t u : list[list.size() - 2].tasks) edges.push_back({u, t});
        }
        list.back().tasks.push_back(t);
      } else {
        if (!list.empty()) {
          for (uint32_t u : list.back().tasks) edges.push_back({u, t});
        }
        list.push_back(Group{m, {t}});
      }
    }
  }

  std::sort(edges.begin(), edges.end());
  edges.erase(std::unique(edges.begin(), edges.end()), edges.end());

  for (int i = 0; i <= ntasks; ++i) row_ptr[i] = 0;
  for (int i = 0; i < ntasks; ++i) indeg[i] = 0;
  for (auto& e : edges) {
    row_ptr[e.first + 1] += 1;
    indeg[e.second] += 1;
  }
  for (int i = 0; i < ntasks; ++i) row_ptr[i + 1] += row_ptr[i];
  const long long ne = (long long)edges.size();
  if (ne <= col_cap && col != nullptr) {
    for (long long i = 0; i < ne; ++i) col[i] = edges[i].second;
  }
  return ne;
}

// ---------------------------------------------------------------------------
// Tile operations, plain FP64 loops.  Tiles are row-major: element (r, c) of
// a tile with leading dimension ld sits at p[r*ld + c].
// ---------------------------------------------------------------------------

// Unblocked Cholesky-Crout, column by column:
//   l_jj = sqrt(a_jj - sum_{k<j} l_jk^2),
//   l_ij = (a_ij - sum_{k<j} l_ik l_jk) / l_jj   for i > j.
// Writes L over the lower triangle (diagonal included); the strict upper
// triangle is not touched.  Returns 0, or the 1-based column whose pivot is
// not positive (or NaN), as LAPACK's info.
int spxo_potrf(double* a, int n, int lda) {
  for (int j = 0; j < n; ++j) {
    double d = a[(size_t)j * lda + j];
    for (int k = 0; k < j; ++k) {
      const double l = a[(size_t)j * lda + k];
      d = d - l * l;
    }
    if (!(d > 0.0)) return j + 1;
    const double ljj = std::sqrt(d);
    a[(size_t)j * lda + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = a[(size_t)i * lda + j];
      for (int k = 0; k < j; ++k) s = s - a[(size_t)i * lda + k] * a[(size_t)j * lda + k];
      a[(size_t)i * lda + j] = s / ljj;
    }
  }
  return 0;
}

// X L^T = A, solved in place row by row (A is m x n, L is n x n lower):
//   x_rj = (a_rj - sum_{k<j} x_rk l_jk) / l_jj.
static void trsm_right_lt(const double* l, int ldl, double* a, int m, int n, int lda) {
  for (int r = 0; r < m; ++r) {
    double* x = a + (size_t)r * lda;
    for (int j = 0; j < n; ++j) {
      double s = x[j];
      for (int k = 0; k < j; ++k) s = s - x[k] * l[(size_t)j * ldl + k];
      x[j] = s / l[(size_t)j * ldl + j];
    }
  }
}

// C <- C - A A^T on the lower triangle (C n x n, A n x k).
static void syrk_lower_sub(const double* a, int lda, double* c, int n, int k, int ldc) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = c[(size_t)i * ldc + j];
      for (int p = 0; p < k; ++p) s = s - a[(size_t)i * lda + p] * a[(size_t)j * lda + p];
      c[(size_t)i * ldc + j] = s;
    }
}

// C <- C - A B^T (C m x n, A m x k, B n x k).
static void gemm_nt_sub(const double* a, int lda, const double* b, int ldb, double* c,
                        int m, int n, int k, int ldc) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) {
      double s = c[(size_t)i * ldc + j];
      for (int p = 0; p < k; ++p) s = s - a[(size_t)i * lda + p] * b[(size_t)j * ldb + p];
      c[(size_t)i * ldc + j] = s;
    }
}

// C <- C + A B (C m x n, A m x k, B k x n), accumulated into c_ij term by term.
static void gemm_nn_add(const double* a, int lda, const double* b, int ldb, double* c,
                        int m, int n, int k, int ldc) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) {
      double s = c[(size_t)i * ldc + j];
      for (int p = 0; p < k; ++p) s = s + a[(size_t)i * lda + p] * b[(size_t)p * ldb + j];
      c[(size_t)i * ldc + j] = s;
    }
}

// Forward substitution L Y = X, in place, for every column of X (n x nrhs).
void spxo_trsv_lower(const double* l, int ldl, double* x, int n, int nrhs, int ldx) {
  for (int c = 0; c < nrhs; ++c)
    for (int i = 0; i < n; ++i) {
      double s = x[(size_t)i * ldx + c];
      for (int k = 0; k < i; ++k) s = s - l[(size_t)i * ldl + k] * x[(size_t)k * ldx + c];
      x[(size_t)i * ldx + c] = s / l[(size_t)i * ldl + i];
    }
}

// Back substitution L^T Y = X, in place.
void spxo_trsv_lower_t(const double* l, int ldl, double* x, int n, int nrhs, int ldx) {
  for (int c = 0; c < nrhs; ++c)
    for (int i = n - 1; i >= 0; --i) {
      double s = x[(size_t)i * ldx + c];
      for (int k = i + 1; k < n; ++k) s = s - l[(size_t)k * ldl + i] * x[(size_t)k * ldx + c];
      x[(size_t)i * ldx + c] = s / l[(size_t)i * ldl + i];
    }
}

// X_i <- X_i - L X_k (X_i m x nrhs, L m x k, X_k k x nrhs).
static void gemm_fwd(const double* l, int ldl, const double* xk, int ldk, double* xi, int ldi,
                     int m, int k, int nrhs) {
  for (int i = 0; i < m; ++i)
    for (int c = 0; c < nrhs; ++c) {
      double s = xi[(size_t)i * ldi + c];
      for (int p = 0; p < k; ++p) s = s - l[(size_t)i * ldl + p] * xk[(size_t)p * ldk + c];
      xi[(size_t)i * ldi + c] = s;
    }
}

// X_i <- X_i - L^T X_k (X_i m x nrhs, L is k x m, X_k k x nrhs).
static void gemm_bwd(const double* l, int ldl, const double* xk, int ldk, double* xi, int ldi,
                     int m, int k, int nrhs) {
  for (int i = 0; i < m; ++i)
    for (int c = 0; c < nrhs; ++c) {
      double s = xi[(size_t)i * ldi + c];
      for (int p = 0; p < k; ++p) s = s - l[(size_t)p * ldl + i] * xk[(size_t)p * ldk + c];
      xi[(size_t)i * ldi + c] = s;
    }
}

// Inverse of a lower-triangular L (n x n): column c of V solves L v = e_c by
// forward substitution (the definition of the inverse, one column at a
// time).  Entries above the diagonal come out zero.
void spxo_trtri(const double* l, int ldl, double* v, int n, int ldv) {
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double s = i == c ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s = s - l[(size_t)i * ldl + k] * v[(size_t)k * ldv + c];
      v[(size_t)i * ldv + c] = s / l[(size_t)i * ldl + i];
    }
}

// Y <- T X or Y <- T^T X (T n x n, X and Y n x nrhs): plain matrix product
// over the whole of T.
static void trmm(const double* t, int ldt, bool trans, const double* x, int ldx, double* y,
                 int ldy, int n, int nrhs) {
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < nrhs; ++c) {
      double s = 0.0;
      for (int k = 0; k < n; ++k)
        s = s + (trans ? t[(size_t)k * ldt + i] : t[(size_t)i * ldt + k]) * x[(size_t)k * ldx + c];
      y[(size_t)i * ldy + c] = s;
    }
}

// A <- A V^T (A m x n, V n x n): plain matrix product over the whole of V,
// one row of A at a time through a copy of the row (the update is in place).
static void trsm_inv(const double* v, int ldv, double* a, int lda, int m, int n) {
  std::vector<double> row(n);
  for (int i = 0; i < m; ++i) {
    for (int k = 0; k < n; ++k) row[k] = a[(size_t)i * lda + k];
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s = s + row[k] * v[(size_t)c * ldv + k];
      a[(size_t)i * lda + c] = s;
    }
  }
}

// Direct Coulomb summation (the paper's particle test case): for each target
// particle i of t (rows x, y, z, q, phi, Ex, Ey, Ez) and each source j of src
// (j != i when both are the same group), with d = x_i - x_j and r = |d| > 0:
//   phi_i += q_j / r,   E_i += q_j d / r^3.
static void nbody_interact(double* t, int ldt, int nt, const double* src, int lds, int ns,
                           bool self) {
  for (int i = 0; i < nt; ++i) {
    double* ti = t + (size_t)i * ldt;
    for (int j = 0; j < ns; ++j) {
      if (self && j == i) continue;
      const double* sj = src + (size_t)j * lds;
      const double dx = ti[0] - sj[0], dy = ti[1] - sj[1], dz = ti[2] - sj[2];
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (!(r2 > 0.0)) continue;
      const double r = std::sqrt(r2);
      const double r3 = r * r * r;
      ti[4] = ti[4] + sj[3] / r;
      ti[5] = ti[5] + sj[3] * dx / r3;
      ti[6] = ti[6] + sj[3] * dy / r3;
      ti[7] = ti[7] + sj[3] * dz / r3;
    }
  }
}

// A tile: base pointer, shape and leading dimension (row-major).
typedef struct {
  double* ptr;
  int rows, cols, ld, pad;
} spxo_tile;

// Run the tasks one after another in insertion order (STF sequential
// semantics).  task_tiles holds 4 tile indices per task in the fixed operand
// order of each op (see the op list above; unused slots are ignored).
// task_arg is the global column offset of a POTRF tile, used for info.
// Returns 0, or 1 when a POTRF meets a non-positive pivot (info set to the
// 1-based global column; later tasks are not run).  -1 on bad input.
int spxo_execute(int ntasks, const int* task_op, const int* task_tiles,
                 const long long* task_arg, const spxo_tile* tiles, int ntiles,
                 int* info) {
  *info = 0;
  for (int t = 0; t < ntasks; ++t) {
    const int* h = task_tiles + 4 * (size_t)t;
    auto tile = [&](int s) -> const spxo_tile& { return tiles[h[s]]; };
    for (int s = 0; s < 3; ++s)
      if (task_op[t] != O_NOP && task_op[t] != O_SPIN && (h[s] < -1 || h[s] >= ntiles)) return -1;
    switch (task_op[t]) {
      case O_POTRF: {
        const spxo_tile& A = tile(0);
        const int r = spxo_potrf(A.ptr, A.rows, A.ld);
        if (r != 0) {
          *info = (int)task_arg[t] + r;
          return 1;
        }
        break;
      }
      case O_TRSM: {
        const spxo_tile& L = tile(0);
        const spxo_tile& A = tile(1);
        trsm_right_lt(L.ptr, L.ld, A.ptr, A.rows, A.cols, A.ld);
        break;
      }
      case O_SYRK: {
        const spxo_tile& L = tile(0);
        const spxo_tile& C = tile(1);
        syrk_lower_sub(L.ptr, L.ld, C.ptr, C.rows, L.cols, C.ld);
        break;
      }
      case O_GEMM_NT_SUB: {
        const spxo_tile& A = tile(0);
        const spxo_tile& B = tile(1);
        const spxo_tile& C = tile(2);
        gemm_nt_sub(A.ptr, A.ld, B.ptr, B.ld, C.ptr, C.rows, C.cols, A.cols, C.ld);
        break;
      }
      case O_GEMM_NN_ADD: {
        const spxo_tile& A = tile(0);
        const spxo_tile& B = tile(1);
        const spxo_tile& C = tile(2);
        gemm_nn_add(A.ptr, A.ld, B.ptr, B.ld, C.ptr, C.rows, C.cols, A.cols, C.ld);
        break;
      }
      case O_TRSM_L_FWD: {
        const spxo_tile& L = tile(0);
        const spxo_tile& X = tile(1);
        spxo_trsv_lower(L.ptr, L.ld, X.ptr, X.rows, X.cols, X.ld);
        break;
      }
      case O_GEMM_FWD: {
        const spxo_tile& L = tile(0);
        const spxo_tile& Xk = tile(1);
        const spxo_tile& Xi = tile(2);
        gemm_fwd(L.ptr, L.ld, Xk.ptr, Xk.ld, Xi.ptr, Xi.ld, Xi.rows, L.cols, Xi.cols);
        break;
      }
      case O_TRSM_LT_BWD: {
        const spxo_tile& L = tile(0);
        const spxo_tile& X = tile(1);
        spxo_trsv_lower_t(L.ptr, L.ld, X.ptr, X.rows, X.cols, X.ld);
        break;
      }
      case O_GEMM_BWD: {
        const spxo_tile& L = tile(0);
        const spxo_tile& Xk = tile(1);
        const spxo_tile& Xi = tile(2);
        gemm_bwd(L.ptr, L.ld, Xk.ptr, Xk.ld, Xi.ptr, Xi.ld, Xi.rows, L.rows, Xi.cols);
        break;
      }
      case O_COPY:
      case O_AXPY: {
        const spxo_tile& X = tile(0);
        const spxo_tile& Y = tile(1);
        for (int r = 0; r < Y.rows; ++r)
          for (int c = 0; c < Y.cols; ++c) {
            const double v = X.ptr[(size_t)r * X.ld + c];
            double& y = Y.ptr[(size_t)r * Y.ld + c];
            y = task_op[t] == O_AXPY ? y + v : v;
          }
        break;
      }
      case O_TRMM: {
        const spxo_tile& Tt = tile(0);
        const spxo_tile& X = tile(1);
        const spxo_tile& Y = tile(2);
        trmm(Tt.ptr, Tt.ld, task_arg[t] != 0, X.ptr, X.ld, Y.ptr, Y.ld, Y.rows, Y.cols);
        break;
      }
      case O_TRTRI: {
        const spxo_tile& L = tile(0);
        const spxo_tile& V = tile(1);
        spxo_trtri(L.ptr, L.ld, V.ptr, L.rows, V.ld);
        break;
      }
      case O_TRSM_INV: {
        const spxo_tile& V = tile(0);
        const spxo_tile& A = tile(1);
        trsm_inv(V.ptr, V.ld, A.ptr, A.ld, A.rows, A.cols);
        break;
      }
      case O_NBODY_SELF: {
        const spxo_tile& P = tile(0);
        nbody_interact(P.ptr, P.ld, P.rows, P.ptr, P.ld, P.rows, true);
        break;
      }
      case O_POTRF_PANEL: {
        const spxo_tile& L = tile(0);
        const spxo_tile& A = tile(1);
        const int r = spxo_potrf(L.ptr, L.rows, L.ld);
        if (r != 0) {
          *info = (int)task_arg[t] + r;
          return 1;
        }
        trsm_right_lt(L.ptr, L.ld, A.ptr, A.rows, A.cols, A.ld);
        break;
      }
      case O_NBODY_PAIR: {
        const spxo_tile& P = tile(0);
        const spxo_tile& Q = tile(1);
        nbody_interact(P.ptr, P.ld, P.rows, Q.ptr, Q.ld, Q.rows, false);
        nbody_interact(Q.ptr, Q.ld, Q.rows, P.ptr, P.ld, P.rows, false);
        break;
      }
      case O_NOP:
      case O_SPIN:
        break;
      default:
        return -1;
    }
  }
  return 0;
}

// The AXPY test case in single precision: y <- y + alpha x over n values,
// piece after piece (the tasks are independent: any order gives the same
// values).  Each value is fl(fl(alpha x) + y), the product skipped when
// alpha = 1; alpha is rounded to FP32 first.
void spxo_axpy_f32(long long n, float alpha, const float* x, float* y) {
  for (long long i = 0; i < n; ++i) y[i] = alpha == 1.0f ? y[i] + x[i] : alpha * x[i] + y[i];
}

// Untiled GEMM C <- C + A B (n x n, row-major, ld = n).
void spxo_gemm_untiled(const double* a, const double* b, double* c, int n) {
  gemm_nn_add(a, n, b, n, c, n, n, n, n);
}

// ---------------------------------------------------------------------------
// Metrics.  Error-free transformations (Knuth TwoSum, FMA-based TwoProduct)
// and the compensated dot product Dot2 of Ogita, Rump and Oishi (2005).
// ---------------------------------------------------------------------------

struct DD {
  double hi, lo;
};

static inline void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

static inline void two_prod(double a, double b, double& p, double& e) {
  p = a * b;
  e = std::fma(a, b, -p);
}

// Accumulator for sum(x_i * y_i) with an error term (Dot2).
struct Dot2 {
  double s = 0.0, c = 0.0;
  inline void add_prod(double x, double y) {
    double p, ep, t, et;
    two_prod(x, y, p, ep);
    two_sum(s, p, t, et);
    s = t;
    c += ep + et;
  }
  inline void add(double x) {
    double t, et;
    two_sum(s, x, t, et);
    s = t;
    c += et;
  }
  inline double value() const { return s + c; }
};

// ||A - L L^T||_F / ||A||_F over the full symmetric matrix (A given in full,
// L = lower triangle of l including the diagonal).
double spxo_factor_backward_error(const double* a, int lda, const double* l, int ldl, int n) {
  long double num = 0.0L, den = 0.0L;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const int lo = std::min(i, j);
      Dot2 d;
      d.add(a[(size_t)i * lda + j]);
      for (int k = 0; k <= lo; ++k) d.add_prod(-l[(size_t)i * ldl + k], l[(size_t)j * ldl + k]);
      const long double r = d.value();
      num += r * r;
      const long double av = a[(size_t)i * lda + j];
      den += av * av;
    }
  return (double)std::sqrt(num / den);
}

// Normwise backward error of each column x of X for A x = b (Rigal-Gaches):
//   eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf).
// A is n x n in full; X and B are n x nrhs row-major with ld = nrhs.
void spxo_solve_backward_error(const double* a, int lda, const double* x, const double* b,
                               int n, int nrhs, double* eta) {
  double anorm = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += std::fabs(a[(size_t)i * lda + j]);
    anorm = std::max(anorm, s);
  }
  for (int c = 0; c < nrhs; ++c) {
    double rmax = 0.0, xmax = 0.0, bmax = 0.0;
    for (int i = 0; i < n; ++i) {
      Dot2 d;
      d.add(b[(size_t)i * nrhs + c]);
      for (int j = 0; j < n; ++j) d.add_prod(-a[(size_t)i * lda + j], x[(size_t)j * nrhs + c]);
      rmax = std::max(rmax, std::fabs(d.value()));
      xmax = std::max(xmax, std::fabs(x[(size_t)i * nrhs + c]));
      bmax = std::max(bmax, std::fabs(b[(size_t)i * nrhs + c]));
    }
    eta[c] = rmax / (anorm * xmax + bmax);
  }
}

// Freivalds-style probe of a factorization, O(n^2):
//   ||A v - L (L^T v)||_2 / (||A||_F ||v||_2)
// for one vector v.  A in full (lda), L = lower triangle of l (ldl).
double spxo_freivalds(const double* a, int lda, const double* l, int ldl, int n, const double* v) {
  std::vector<double> w(n), av(n);
  for (int k = 0; k < n; ++k) {  // w = L^T v
    Dot2 d;
    for (int i = k; i < n; ++i) d.add_prod(l[(size_t)i * ldl + k], v[i]);
    w[k] = d.value();
  }
  long double num = 0.0L, afro = 0.0L, vn = 0.0L;
  for (int i = 0; i < n; ++i) {
    Dot2 d;
    for (int j = 0; j < n; ++j) {
      d.add_prod(a[(size_t)i * lda + j], v[j]);
      const long double x = a[(size_t)i * lda + j];
      afro += x * x;
    }
    for (int k = 0; k <= i; ++k) d.add_prod(-l[(size_t)i * ldl + k], w[k]);
    const long double r = d.value();
    num += r * r;
    vn += (long double)v[i] * v[i];
  }
  return (double)(std::sqrt(num) / (std::sqrt(afro) * std::sqrt(vn)));
}

int spxo_abi_version(void) { return 1; }

}  // extern "C"
