// Task-graph builders for the paper's workloads (section "Numerical
// applications"), written on top of the public insertion calls so that a
// whole graph is inserted in one C call:
//   * tiled Cholesky A = L L^T with POTRF, TRSM, SYRK and GEMM tasks,
//     right-looking, k outer, optionally followed by the block forward and
//     back solves of A Y = X;
//   * tiled GEMM C += A B with one task per (i, j, k) that depends on the
//     block C_ij it updates;
//   * the inverses of the diagonal factor tiles (TRTRI) and the block solve
//     that applies them as products (TRMM), for refinement;
//   * the scheduler-overhead pattern of the paper's engine benchmark: chains
//     of tasks that only wait.
#include <chrono>
#include <cstdint>
#include <initializer_list>
#include <vector>

#include <cuda_runtime.h>

#include "spx.h"

namespace {

struct Tiles {
  int T = 0, b = 0;
  std::vector<unsigned> h;
  unsigned& at(int i, int j) { return h[(size_t)i * T + j]; }
};

int register_tiles(spx_graph_t g, double* base, int n_rows, int n_cols, int ld, int b,
                   bool lower_only, Tiles& out, char* lowp = nullptr, int ldlo = 0, int elem = 0) {
  const int Tr = (n_rows + b - 1) / b, Tc = (n_cols + b - 1) / b;
  out.T = Tr > Tc ? Tr : Tc;
  out.b = b;
  out.h.assign((size_t)out.T * out.T, 0xFFFFFFFFu);
  for (int i = 0; i < Tr; ++i)
    for (int j = 0; j < Tc; ++j) {
      if (lower_only && j > i) continue;
      const int r = n_rows - i * b < b ? n_rows - i * b : b;
      const int c = n_cols - j * b < b ? n_cols - j * b : b;
      void* lo = lowp ? lowp + ((size_t)i * b * ldlo + (size_t)j * b) * elem : nullptr;
      int rc = spx_tile_register(g, base + (size_t)i * b * ld + (size_t)j * b, r, c, ld, SPX_DT_F64,
                                 lo, lo ? ldlo : 0, &out.at(i, j));
      if (rc != SPX_OK) return rc;
    }
  return SPX_OK;
}

}  // namespace

namespace {

// factor: insert the factorization tasks; dev_X: the solve tasks too;
// dev_V (mixed precision only): the panel solves as TRTRI + TRSM_INV.
// Tiles of the lower triangle of A whose off-diagonal tiles (i, k) own split
// slot i (i - 1) / 2 + k of the store at S (SPX_F64_OZAKI); with inverse
// panels (inv) the diagonal inverses V_k own slots T (T - 1) / 2 + k.
int register_ozaki_tiles(spx_graph_t g, double* A, int n, int lda, int b, char* S,
                         long long S_bytes, Tiles& out, bool inv) {
  const long long slot = spx_ozaki_slot_bytes(b);
  const int T = (n + b - 1) / b;
  const long long nslots = (long long)T * (T - 1) / 2 + (inv ? T : 0);
  if (!slot || !S || ((uintptr_t)S & 255)) return SPX_ERR_INVALID_ARG;
  if (nslots > 0) {
    if (S_bytes < nslots * slot || nslots > 0x7FFFFFFF) return SPX_ERR_INVALID_ARG;
    const int rc = spx_ozaki_register(g, S, (int)nslots, b, nullptr);
    if (rc != SPX_OK) return rc;
  }
  out.T = T;
  out.b = b;
  out.h.assign((size_t)T * T, 0xFFFFFFFFu);
  for (int i = 0; i < T; ++i)
    for (int j = 0; j <= i; ++j) {
      const int r = n - i * b < b ? n - i * b : b;
      const int c = n - j * b < b ? n - j * b : b;
      char* lo = i > j ? S + ((long long)i * (i - 1) / 2 + j) * slot : nullptr;
      const int rc = spx_tile_register(g, A + (size_t)i * b * lda + (size_t)j * b, r, c, lda,
                                       SPX_DT_F64, lo, lo ? b : 0, &out.at(i, j));
      if (rc != SPX_OK) return rc;
    }
  return SPX_OK;
}

int insert_cholesky(spx_graph_t g, double* dev_A, int n, int lda, int b, void* dev_Alo, int ldlo,
                    bool factor, double* dev_X, int nrhs, int ldx, int lookahead, int prec,
                    long long* out_ntasks, double* dev_V = nullptr, int ldv = 0,
                    long long S_bytes = 0, bool fuse = false) {
  if (!g || !dev_A || n < 1 || b < 1 || lda < n || (dev_X && (nrhs < 1 || ldx < nrhs)))
    return SPX_ERR_INVALID_ARG;
  const bool oz = prec == SPX_F64_OZAKI;
  if (prec != SPX_F64 && !oz && (!dev_Alo || ldlo < n)) return SPX_ERR_INVALID_ARG;
  if (dev_V && (prec == SPX_F64 || ldv < (b < n ? b : n))) return SPX_ERR_INVALID_ARG;
  const int elem = prec == SPX_BF16 ? 2 : 4;
  int rc = SPX_OK;
  if (prec != SPX_F64 && !oz)
    rc = spx_lowp_register(g, dev_Alo, n, n, ldlo, prec == SPX_BF16 ? SPX_DT_BF16 : SPX_DT_F32,
                           nullptr);
  if (rc != SPX_OK) return rc;
  Tiles A;
  if (oz)
    rc = register_ozaki_tiles(g, dev_A, n, lda, b, (char*)dev_Alo, S_bytes, A, dev_V != nullptr);
  else
    rc = register_tiles(g, dev_A, n, n, lda, b, true, A,
                        prec != SPX_F64 ? (char*)dev_Alo : nullptr, ldlo, elem);
  if (rc != SPX_OK) return rc;
  const int T = A.T;
  const int R = SPX_READ, W = SPX_WRITE;
  const int hi = lookahead ? 1 : 0;
  const int crit = lookahead ? 2 : 0;  // critical path: high priority, finer parts
  long long count = 0;
  // lookahead >= 2 (small problems, where the whole DAG is one chain): every
  // task on the critical-path queue, cut into the finer parts
  auto ins = [&](int op, std::initializer_list<unsigned> hs, std::initializer_list<int> ms,
                 int prio, unsigned* id, int p = SPX_F64) {
    const unsigned* hp = hs.begin();
    const int* mp = ms.begin();
    int r = spx_task_insert(g, op, hp, mp, (int)hs.size(), lookahead >= 2 ? 2 : prio, p, id);
    if (r == SPX_OK) ++count;
    return r;
  };
  for (int k = 0; k < T && rc == SPX_OK && factor; ++k) {
    unsigned t = 0;
    // fuse: POTRF(k) and the solve of the critical panel tile (k+1, k) as one
    // task (POTRF_PANEL), the rest of the panel as below
    const bool fused = fuse && k + 1 < T;
    if (fused)
      rc = ins(SPX_OP_POTRF_PANEL, {A.at(k, k), A.at(k + 1, k)}, {W, W}, crit, &t, prec);
    else
      rc = ins(SPX_OP_POTRF, {A.at(k, k)}, {W}, crit, &t, SPX_F64);
    if (rc == SPX_OK) rc = spx_task_set_arg(g, t, (long long)k * b);
    if (dev_V) {
      // The panel below the critical one: V_k <- L_kk^{-1} (FP64), then
      // A_ik <- A_ik V_k^T on the tensor cores.  The critical panel tile
      // (k+1, k) is solved by FP64 substitution straight after POTRF, so the
      // inversion stays off the critical path.
      const int bk = n - k * b < b ? n - k * b : b;
      unsigned v = 0;
      if (rc == SPX_OK && k + 1 < T && !fused)
        rc = ins(SPX_OP_TRSM, {A.at(k, k), A.at(k + 1, k)}, {R, W}, crit, nullptr, prec);
      // split prec: V_k owns a slot after the factor tiles' and is split
      // after the inversion (the TRSM_INV products read its digits)
      char* vslot = oz ? (char*)dev_Alo + ((long long)T * (T - 1) / 2 + k) *
                                              spx_ozaki_slot_bytes(b)
                       : nullptr;
      if (rc == SPX_OK)
        rc = spx_tile_register(g, dev_V + (size_t)k * b * ldv, bk, bk, ldv, SPX_DT_F64, vslot,
                               oz ? b : 0, &v);
      if (rc == SPX_OK)
        rc = ins(SPX_OP_TRTRI, {A.at(k, k), v}, {R, W}, hi, nullptr, oz ? prec : SPX_F64);
      for (int i = k + 2; i < T && rc == SPX_OK; ++i)
        rc = ins(SPX_OP_TRSM_INV, {v, A.at(i, k)}, {R, W}, hi, nullptr, prec);
    }
    for (int i = k + (fused ? 2 : 1); i < T && rc == SPX_OK && !dev_V; ++i)
      rc = ins(SPX_OP_TRSM, {A.at(k, k), A.at(i, k)}, {R, W}, i == k + 1 ? crit : hi, nullptr,
               prec);
    for (int i = k + 1; i < T && rc == SPX_OK; ++i)
      rc = ins(SPX_OP_SYRK, {A.at(i, k), A.at(i, i)}, {R, W}, i == k + 1 ? crit : hi, nullptr,
               prec);
    for (int j = k + 1; j < T && rc == SPX_OK; ++j)
      for (int i = j + 1; i < T && rc == SPX_OK; ++i)
        rc = ins(SPX_OP_GEMM_NT_SUB, {A.at(i, k), A.at(j, k), A.at(i, j)}, {R, R, W},
                 j == k + 1 ? (i == k + 2 ? crit : hi) : 0, nullptr, prec);
  }
  if (rc == SPX_OK && dev_X) {
    std::vector<unsigned> x(T);
    for (int i = 0; i < T && rc == SPX_OK; ++i) {
      const int r = n - i * b < b ? n - i * b : b;
      rc = spx_tile_register(g, dev_X + (size_t)i * b * ldx, r, nrhs, ldx, SPX_DT_F64, nullptr, 0,
                             &x[i]);
    }
    for (int k = 0; k < T && rc == SPX_OK; ++k) {
      rc = ins(SPX_OP_TRSM_L_FWD, {A.at(k, k), x[k]}, {R, W}, hi, nullptr);
      for (int i = k + 1; i < T && rc == SPX_OK; ++i)
        rc = ins(SPX_OP_GEMM_FWD, {A.at(i, k), x[k], x[i]}, {R, R, W}, i == k + 1 ? hi : 0,
                 nullptr);
    }
    for (int k = T - 1; k >= 0 && rc == SPX_OK; --k) {
      rc = ins(SPX_OP_TRSM_LT_BWD, {A.at(k, k), x[k]}, {R, W}, hi, nullptr);
      for (int i = k - 1; i >= 0 && rc == SPX_OK; --i)
        rc = ins(SPX_OP_GEMM_BWD, {A.at(k, i), x[k], x[i]}, {R, R, W}, i == k - 1 ? hi : 0,
                 nullptr);
    }
  }
  if (out_ntasks) *out_ntasks = count;
  return rc;
}

}  // namespace

extern "C" int spx_cholesky_insert(spx_graph_t g, double* dev_A, int n, int lda, int b,
                                   double* dev_X, int nrhs, int ldx, int lookahead, int prec,
                                   long long* out_ntasks) {
  if (prec != SPX_F64) return SPX_ERR_INVALID_ARG;
  return insert_cholesky(g, dev_A, n, lda, b, nullptr, 0, true, dev_X, nrhs, ldx, lookahead,
                         SPX_F64, out_ntasks);
}

extern "C" int spx_cholesky_insert_mixed(spx_graph_t g, double* dev_A, int n, int lda, int b,
                                         void* dev_Alo, int ldlo, double* dev_X, int nrhs, int ldx,
                                         int lookahead, int prec, long long* out_ntasks) {
  if (prec != SPX_TF32 && prec != SPX_BF16) return SPX_ERR_INVALID_ARG;
  return insert_cholesky(g, dev_A, n, lda, b, dev_Alo, ldlo, true, dev_X, nrhs, ldx, lookahead,
                         prec, out_ntasks);
}

extern "C" int spx_cholesky_insert_mixed_inv(spx_graph_t g, double* dev_A, int n, int lda, int b,
                                             void* dev_Alo, int ldlo, double* dev_V, int ldv,
                                             double* dev_X, int nrhs, int ldx, int lookahead,
                                             int prec, long long* out_ntasks) {
  if ((prec != SPX_TF32 && prec != SPX_BF16) || !dev_V) return SPX_ERR_INVALID_ARG;
  return insert_cholesky(g, dev_A, n, lda, b, dev_Alo, ldlo, true, dev_X, nrhs, ldx, lookahead,
                         prec, out_ntasks, dev_V, ldv);
}

extern "C" int spx_cholesky_insert_ozaki(spx_graph_t g, double* dev_A, int n, int lda, int b,
                                         void* dev_S, long long S_bytes, double* dev_V, int ldv,
                                         int fuse_panel, double* dev_X, int nrhs, int ldx,
                                         int lookahead, long long* out_ntasks) {
  if (!spx_ozaki_slot_bytes(b) || fuse_panel < 0 || fuse_panel > 1) return SPX_ERR_INVALID_ARG;
  return insert_cholesky(g, dev_A, n, lda, b, dev_S, 0, true, dev_X, nrhs, ldx, lookahead,
                         SPX_F64_OZAKI, out_ntasks, dev_V, ldv, S_bytes, fuse_panel != 0);
}

extern "C" int spx_cholesky_host_ozaki(spx_graph_t g, const double* host_A, double* host_L,
                                       int n, int ld_host, int b, double* dev_A, int lda,
                                       void* dev_S, long long S_bytes, double* dev_V, int ldv,
                                       void* stream, int* info) {
  if (info) *info = 0;
  if (!g || !host_A || !host_L || !dev_A || !dev_V || n < 1 || ld_host < n || lda < n ||
      !spx_ozaki_slot_bytes(b) || ldv < (b < n ? b : n))
    return SPX_ERR_INVALID_ARG;
  Tiles A;
  int rc = register_ozaki_tiles(g, dev_A, n, lda, b, (char*)dev_S, S_bytes, A, true);
  if (rc != SPX_OK) return rc;
  const int T = A.T;
  const long long slot = spx_ozaki_slot_bytes(b);
  std::vector<unsigned> V(T);
  for (int k = 0; k < T && rc == SPX_OK; ++k) {  // V_k owns slot T (T - 1) / 2 + k
    const int bk = n - k * b < b ? n - k * b : b;
    rc = spx_tile_register(g, dev_V + (size_t)k * b * ldv, bk, bk, ldv, SPX_DT_F64,
                           (char*)dev_S + ((long long)T * (T - 1) / 2 + k) * slot, b, &V[k]);
  }
  if (rc != SPX_OK) return rc;
  // the task list of spx_cholesky_insert_ozaki (inverse panels, look-ahead
  // marks), its first step ordered by column so that column block j's tasks
  // follow its upload (same accesses per tile in the same order: same DAG)
  long long tasks = T;
  for (int k = 0; k < T; ++k) {
    const long long r = T - k - 1;
    tasks += 1 + (r > 0 ? 1 : 0) + (r > 1 ? r - 1 : 0) + r + r * (r - 1) / 2;
  }
  const long long cap = tasks + (long long)T * T + 64;  // relays
  const int R = SPX_READ, W = SPX_WRITE, P = SPX_F64_OZAKI;
  auto ins = [&](int op, std::initializer_list<unsigned> hs, std::initializer_list<int> ms,
                 int prio, int prec, unsigned* id = nullptr) {
    return spx_task_insert(g, op, hs.begin(), ms.begin(), (int)hs.size(), prio, prec, id);
  };
  // the last writers of column block k: POTRF(k), its panel's solve and products
  std::vector<std::vector<unsigned>> last(T);
  auto head = [&](int k) {  // POTRF, critical solve, inversion, inverse panel products
    unsigned t = 0;
    int r = ins(SPX_OP_POTRF, {A.at(k, k)}, {W}, 2, SPX_F64, &t);
    if (r == SPX_OK) last[k].push_back(t);
    if (r == SPX_OK) r = spx_task_set_arg(g, t, (long long)k * b);
    if (r == SPX_OK && k + 1 < T) {
      r = ins(SPX_OP_TRSM, {A.at(k, k), A.at(k + 1, k)}, {R, W}, 2, P, &t);
      if (r == SPX_OK) last[k].push_back(t);
    }
    if (r == SPX_OK) r = ins(SPX_OP_TRTRI, {A.at(k, k), V[k]}, {R, W}, 1, P);
    for (int i = k + 2; i < T && r == SPX_OK; ++i) {
      r = ins(SPX_OP_TRSM_INV, {V[k], A.at(i, k)}, {R, W}, 1, P, &t);
      if (r == SPX_OK) last[k].push_back(t);
    }
    return r;
  };
  auto update = [&](int k, int j) {  // SYRK(j, k) and the GEMMs of column j
    int r = ins(SPX_OP_SYRK, {A.at(j, k), A.at(j, j)}, {R, W}, j == k + 1 ? 2 : 1, P);
    for (int i = j + 1; i < T && r == SPX_OK; ++i)
      r = ins(SPX_OP_GEMM_NT_SUB, {A.at(i, k), A.at(j, k), A.at(i, j)}, {R, R, W},
              j == k + 1 ? (i == k + 2 ? 2 : 1) : 0, P);
    return r;
  };
  // column block 0 on the launch stream, ahead of the kernel; its tasks (split
  // prec: they fix the kernel family) inserted before the stream begins
  const int w0 = n < b ? n : b;
  rc = spx_copy2d(dev_A, (size_t)lda * 8, host_A, (size_t)ld_host * 8, (size_t)w0 * 8, (size_t)n,
                  stream);
  if (rc == SPX_OK) rc = head(0);
  if (rc == SPX_OK)
    rc = spx_stream_begin(g, stream, (int)cap, (int)(T * (T + 1) / 2 + T), 3 * cap, 16 * cap);
  if (rc != SPX_OK) return rc;
  for (int j = 1; j < T && rc == SPX_OK; ++j) {  // upload column block j, then its step-0 tasks
    const int c0 = j * b, w = n - c0 < b ? n - c0 : b;
    rc = spx_stream_copy_h2d(g, dev_A + (size_t)c0 * lda + c0, (size_t)lda * 8,
                             host_A + (size_t)c0 * ld_host + c0, (size_t)ld_host * 8,
                             (size_t)w * 8, (size_t)(n - c0));
    if (rc == SPX_OK) rc = update(0, j);
    if (rc == SPX_OK) rc = spx_stream_flush(g);
  }
  for (int k = 1; k < T && rc == SPX_OK; ++k) {
    rc = head(k);
    for (int j = k + 1; j < T && rc == SPX_OK; ++j) rc = update(k, j);
    if (rc == SPX_OK) rc = spx_stream_flush(g);
  }
  const int end_rc = spx_stream_end(g);
  // the factor's column blocks back to the host, each as soon as its last
  // writers have finished (copy engine, beside the running kernel)
  cudaStream_t down = nullptr;
  if (cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking) != cudaSuccess) down = nullptr;
  int next = 0, copy_rc = SPX_OK;
  auto download = [&](int j) {
    const int c0 = j * b, w = n - c0 < b ? n - c0 : b;
    const int e = spx_copy2d(host_L + (size_t)c0 * ld_host + c0, (size_t)ld_host * 8,
                             dev_A + (size_t)c0 * lda + c0, (size_t)lda * 8, (size_t)w * 8,
                             (size_t)(n - c0), down ? (void*)down : stream);
    if (copy_rc == SPX_OK) copy_rc = e;
  };
  int wrc = SPX_ERR_TIMEOUT;
  bool finished = false;
  auto since = std::chrono::steady_clock::now();
  while (rc == SPX_OK && end_rc == SPX_OK && down) {
    std::vector<int> done;
    while (next < T) {
      done.assign(last[next].size(), 0);
      if (spx_graph_tasks_done(g, last[next].data(), (int)last[next].size(), done.data()) != SPX_OK)
        break;
      bool all = true;
      for (int d : done) all = all && d;
      if (!all) break;
      download(next++);
      since = std::chrono::steady_clock::now();
    }
    if (next == T) break;
    wrc = spx_graph_wait(g, 200000, info);  // a 0.2 ms pause, or the run's end
    if (wrc != SPX_ERR_TIMEOUT) {
      finished = true;
      break;
    }
    // a device watchdog also answers SPX_ERR_TIMEOUT: stop polling when no
    // column has finished for a long time and wait for the status below
    if (std::chrono::steady_clock::now() - since > std::chrono::seconds(30)) break;
  }
  if (!finished) wrc = spx_graph_wait(g, 0, info);
  if (rc == SPX_OK) rc = end_rc;
  if (rc == SPX_OK) rc = wrc;
  if (rc == SPX_OK || rc == SPX_NOT_SPD)
    while (next < T) download(next++);
  const bool synced = (!down || cudaStreamSynchronize(down) == cudaSuccess) &&
                      cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess;
  if (down) cudaStreamDestroy(down);
  if (rc != SPX_OK && rc != SPX_NOT_SPD) return rc;
  if (copy_rc != SPX_OK) return copy_rc;
  return synced ? rc : SPX_ERR_CUDA;
}

extern "C" int spx_solve_insert(spx_graph_t g, double* dev_L, int n, int ld, int b,
                                double* dev_X, int nrhs, int ldx, long long* out_ntasks) {
  if (!dev_X) return SPX_ERR_INVALID_ARG;
  return insert_cholesky(g, dev_L, n, ld, b, nullptr, 0, false, dev_X, nrhs, ldx, 1, SPX_F64,
                         out_ntasks);
}

namespace {

// Square b_k x b_k blocks stacked in an n x b matrix (row block k at row
// k*b): the inverses of the diagonal factor tiles.
size_t dt_bytes(int dtype) { return dtype == SPX_DT_F32 ? 4 : 8; }

int register_diag_blocks(spx_graph_t g, void* base, int n, int ld, int b,
                         std::vector<unsigned>& out, int dtype = SPX_DT_F64) {
  const int T = (n + b - 1) / b;
  out.assign(T, 0);
  for (int k = 0; k < T; ++k) {
    const int r = n - k * b < b ? n - k * b : b;
    char* p = (char*)base + (size_t)k * b * ld * dt_bytes(dtype);
    const int rc = spx_tile_register(g, p, r, r, ld, dtype, nullptr, 0, &out[k]);
    if (rc != SPX_OK) return rc;
  }
  return SPX_OK;
}

// Row blocks (b_k x nrhs) of an n x nrhs right-hand side.
int register_row_blocks(spx_graph_t g, void* base, int n, int nrhs, int ld, int b,
                        std::vector<unsigned>& out, int dtype = SPX_DT_F64) {
  const int T = (n + b - 1) / b;
  out.assign(T, 0);
  for (int k = 0; k < T; ++k) {
    const int r = n - k * b < b ? n - k * b : b;
    char* p = (char*)base + (size_t)k * b * ld * dt_bytes(dtype);
    const int rc = spx_tile_register(g, p, r, nrhs, ld, dtype, nullptr, 0, &out[k]);
    if (rc != SPX_OK) return rc;
  }
  return SPX_OK;
}

}  // namespace

extern "C" int spx_trtri_insert(spx_graph_t g, double* dev_L, int n, int ldl, int b,
                                double* dev_V, int ldv, long long* out_ntasks) {
  if (!g || !dev_L || !dev_V || n < 1 || b < 1 || ldl < n || ldv < (b < n ? b : n))
    return SPX_ERR_INVALID_ARG;
  Tiles L;
  std::vector<unsigned> V;
  int rc = register_tiles(g, dev_L, n, n, ldl, b, true, L);
  if (rc == SPX_OK) rc = register_diag_blocks(g, dev_V, n, ldv, b, V);
  long long count = 0;
  const int R = SPX_READ, W = SPX_WRITE;
  for (int k = 0; k < L.T && rc == SPX_OK; ++k) {
    const unsigned hs[2] = {L.at(k, k), V[k]};
    const int ms[2] = {R, W};
    rc = spx_task_insert(g, SPX_OP_TRTRI, hs, ms, 2, 0, SPX_F64, nullptr);
    if (rc == SPX_OK) ++count;
  }
  if (out_ntasks) *out_ntasks = count;
  return rc;
}

extern "C" int spx_solve_inv_insert(spx_graph_t g, double* dev_L, int n, int ldl, int b,
                                    double* dev_V, int ldv, double* dev_R, double* dev_D,
                                    int nrhs, int ldx, long long* out_ntasks) {
  if (!g || !dev_L || !dev_V || !dev_R || !dev_D || dev_R == dev_D || n < 1 || b < 1 ||
      ldl < n || ldv < (b < n ? b : n) || nrhs < 1 || ldx < nrhs)
    return SPX_ERR_INVALID_ARG;
  Tiles L;
  std::vector<unsigned> V, Rb, Db;
  int rc = register_tiles(g, dev_L, n, n, ldl, b, true, L);
  if (rc == SPX_OK) rc = register_diag_blocks(g, dev_V, n, ldv, b, V);
  if (rc == SPX_OK) rc = register_row_blocks(g, dev_R, n, nrhs, ldx, b, Rb);
  if (rc == SPX_OK) rc = register_row_blocks(g, dev_D, n, nrhs, ldx, b, Db);
  const int R = SPX_READ, W = SPX_WRITE, T = L.T;
  long long count = 0;
  auto ins = [&](int op, unsigned h0, unsigned h1, unsigned h2, int prio, long long arg) {
    const unsigned hs[3] = {h0, h1, h2};
    const int ms[3] = {R, R, W};
    unsigned id = 0;
    int r = spx_task_insert(g, op, hs, ms, 3, prio, SPX_F64, &id);
    if (r == SPX_OK && arg) r = spx_task_set_arg(g, id, arg);
    if (r == SPX_OK) ++count;
    return r;
  };
  // forward: D_k = V_k (R_k - sum_{j<k} L_kj D_j)
  for (int k = 0; k < T && rc == SPX_OK; ++k) {
    rc = ins(SPX_OP_TRMM, V[k], Rb[k], Db[k], 1, 0);
    for (int i = k + 1; i < T && rc == SPX_OK; ++i)
      rc = ins(SPX_OP_GEMM_FWD, L.at(i, k), Db[k], Rb[i], i == k + 1 ? 1 : 0, 0);
  }
  // backward: R_k = V_k^T (D_k - sum_{i>k} L_ik^T R_i)
  for (int k = T - 1; k >= 0 && rc == SPX_OK; --k) {
    rc = ins(SPX_OP_TRMM, V[k], Db[k], Rb[k], 1, 1);
    for (int i = k - 1; i >= 0 && rc == SPX_OK; --i)
      rc = ins(SPX_OP_GEMM_BWD, L.at(k, i), Rb[k], Db[i], i == k - 1 ? 1 : 0, 0);
  }
  if (out_ntasks) *out_ntasks = count;
  return rc;
}

extern "C" int spx_solve_inv_f32_insert(spx_graph_t g, const float* dev_L32, int n, int ldl,
                                        int b, const float* dev_V32, int ldv, const double* dev_R,
                                        float* dev_R32, float* dev_D32, double* dev_X, int nrhs,
                                        int ldx, long long* out_ntasks) {
  if (!g || !dev_L32 || !dev_V32 || !dev_R || !dev_R32 || !dev_D32 || !dev_X ||
      dev_R32 == dev_D32 || (const void*)dev_R == (const void*)dev_X || n < 1 || b < 1 ||
      ldl < n || ldv < (b < n ? b : n) || nrhs < 1 || nrhs > 16 || ldx < nrhs)
    return SPX_ERR_INVALID_ARG;
  const int T = (n + b - 1) / b;
  Tiles L;
  L.T = T;
  L.b = b;
  L.h.assign((size_t)T * T, 0xFFFFFFFFu);
  int rc = SPX_OK;
  for (int i = 0; i < T && rc == SPX_OK; ++i)
    for (int j = 0; j < i && rc == SPX_OK; ++j) {  // strictly lower tiles (the updates' operands)
      const int r = n - i * b < b ? n - i * b : b, c = b;
      rc = spx_tile_register(g, (void*)(dev_L32 + (size_t)i * b * ldl + (size_t)j * b), r, c, ldl,
                             SPX_DT_F32, nullptr, 0, &L.at(i, j));
    }
  std::vector<unsigned> V, R64, X64, Rb, Db;
  if (rc == SPX_OK) rc = register_diag_blocks(g, (void*)dev_V32, n, ldv, b, V, SPX_DT_F32);
  if (rc == SPX_OK) rc = register_row_blocks(g, (void*)dev_R, n, nrhs, ldx, b, R64);
  if (rc == SPX_OK) rc = register_row_blocks(g, dev_X, n, nrhs, ldx, b, X64);
  if (rc == SPX_OK) rc = register_row_blocks(g, dev_R32, n, nrhs, ldx, b, Rb, SPX_DT_F32);
  if (rc == SPX_OK) rc = register_row_blocks(g, dev_D32, n, nrhs, ldx, b, Db, SPX_DT_F32);
  long long count = 0;
  auto ins = [&](int op, const unsigned* hs, int nh, int prio, long long arg) {
    int ms[3] = {SPX_READ, SPX_READ, SPX_READ};
    ms[nh - 1] = SPX_WRITE;
    unsigned id = 0;
    int r = spx_task_insert(g, op, hs, ms, nh, prio, SPX_F64, &id);
    if (r == SPX_OK && arg) r = spx_task_set_arg(g, id, arg);
    if (r == SPX_OK) ++count;
    return r;
  };
  // r (FP64) rounded to FP32
  for (int k = 0; k < T && rc == SPX_OK; ++k) {
    const unsigned hs[2] = {R64[k], Rb[k]};
    rc = ins(SPX_OP_COPY, hs, 2, k == 0 ? 1 : 0, 0);
  }
  // the block solve of spx_solve_inv_insert on the FP32 copies
  for (int k = 0; k < T && rc == SPX_OK; ++k) {
    const unsigned hd[3] = {V[k], Rb[k], Db[k]};
    rc = ins(SPX_OP_TRMM, hd, 3, 1, 0);
    for (int i = k + 1; i < T && rc == SPX_OK; ++i) {
      const unsigned hu[3] = {L.at(i, k), Db[k], Rb[i]};
      rc = ins(SPX_OP_GEMM_FWD, hu, 3, i == k + 1 ? 1 : 0, 0);
    }
  }
  for (int k = T - 1; k >= 0 && rc == SPX_OK; --k) {
    const unsigned hd[3] = {V[k], Db[k], Rb[k]};
    rc = ins(SPX_OP_TRMM, hd, 3, 1, 1);
    for (int i = k - 1; i >= 0 && rc == SPX_OK; --i) {
      const unsigned hu[3] = {L.at(k, i), Rb[k], Db[i]};
      rc = ins(SPX_OP_GEMM_BWD, hu, 3, i == k - 1 ? 1 : 0, 0);
    }
  }
  // x += d (FP32 correction widened exactly)
  for (int k = 0; k < T && rc == SPX_OK; ++k) {
    const unsigned hs[2] = {Rb[k], X64[k]};
    rc = ins(SPX_OP_AXPY, hs, 2, 0, 0);
  }
  if (out_ntasks) *out_ntasks = count;
  return rc;
}

extern "C" int spx_overhead_insert(spx_graph_t g, int chains, int ntasks, int deps,
                                   int commutative, long long spin_ns, long long* out_ntasks) {
  if (!g || chains < 1 || ntasks < 1 || deps < 1 || deps > 16 || spin_ns < 0)
    return SPX_ERR_INVALID_ARG;
  // chains x deps data objects at addresses that are never dereferenced (NOP
  // and SPIN tasks do not touch their tiles)
  const uintptr_t base = (uintptr_t)0x7e0000000000ull;
  std::vector<unsigned> h((size_t)chains * deps);
  int rc = SPX_OK;
  for (size_t i = 0; i < h.size() && rc == SPX_OK; ++i)
    rc = spx_tile_register(g, (void*)(base + 4096 * i), 8, 8, 8, SPX_DT_F64, nullptr, 0, &h[i]);
  const int mode = commutative ? SPX_COMMUTATIVE_WRITE : SPX_WRITE;
  std::vector<int> modes(deps, mode);
  const int op = spin_ns > 0 ? SPX_OP_SPIN : SPX_OP_NOP;
  long long count = 0;
  for (int j = 0; j < ntasks && rc == SPX_OK; ++j)
    for (int c = 0; c < chains && rc == SPX_OK; ++c) {
      unsigned id = 0;
      rc = spx_task_insert(g, op, &h[(size_t)c * deps], modes.data(), deps, 0, SPX_F64, &id);
      if (rc == SPX_OK && spin_ns > 0) rc = spx_task_set_arg(g, id, spin_ns);
      if (rc == SPX_OK) ++count;
    }
  if (out_ntasks) *out_ntasks = count;
  return rc;
}

extern "C" int spx_refine_inv_insert(spx_graph_t g, double* dev_A0, int n, int lda, double* dev_L,
                                     int ldl, int b, double* dev_V, int ldv, double* dev_B,
                                     double* dev_X, double* dev_R, double* dev_D, int nrhs, int ldx,
                                     int sweeps, long long* out_ntasks) {
  if (!g || !dev_A0 || !dev_L || !dev_V || !dev_B || !dev_X || !dev_R || !dev_D || n < 1 ||
      b < 1 || lda < n || ldl < n || ldv < (b < n ? b : n) || nrhs < 1 || ldx < nrhs ||
      sweeps < 0 || dev_R == dev_D)
    return SPX_ERR_INVALID_ARG;
  Tiles A0, L;
  std::vector<unsigned> V, xb, xx, xr, xd;
  int rc = register_tiles(g, dev_A0, n, n, lda, b, false, A0);
  if (rc == SPX_OK) rc = register_tiles(g, dev_L, n, n, ldl, b, true, L);
  if (rc == SPX_OK) rc = register_diag_blocks(g, dev_V, n, ldv, b, V);
  if (rc == SPX_OK) rc = register_row_blocks(g, dev_B, n, nrhs, ldx, b, xb);
  if (rc == SPX_OK) rc = register_row_blocks(g, dev_X, n, nrhs, ldx, b, xx);
  if (rc == SPX_OK) rc = register_row_blocks(g, dev_R, n, nrhs, ldx, b, xr);
  if (rc == SPX_OK) rc = register_row_blocks(g, dev_D, n, nrhs, ldx, b, xd);
  if (rc != SPX_OK) return rc;
  const int T = A0.T, R = SPX_READ, W = SPX_WRITE;
  long long count = 0;
  auto ins = [&](int op, std::initializer_list<unsigned> hs, std::initializer_list<int> ms,
                 int prio, long long arg) {
    unsigned id = 0;
    int r = spx_task_insert(g, op, hs.begin(), ms.begin(), (int)hs.size(), prio, SPX_F64, &id);
    if (r == SPX_OK && arg) r = spx_task_set_arg(g, id, arg);
    if (r == SPX_OK) ++count;
    return r;
  };
  for (int k = 0; k < T && rc == SPX_OK; ++k)
    rc = ins(SPX_OP_TRTRI, {L.at(k, k), V[k]}, {R, W}, 1, 0);
  for (int sw = 0; sw < sweeps && rc == SPX_OK; ++sw) {
    // r = b - A0 x
    for (int i = 0; i < T && rc == SPX_OK; ++i) rc = ins(SPX_OP_COPY, {xb[i], xr[i]}, {R, W}, 0, 0);
    for (int i = 0; i < T && rc == SPX_OK; ++i)
      for (int j = 0; j < T && rc == SPX_OK; ++j)
        rc = ins(SPX_OP_GEMM_FWD, {A0.at(i, j), xx[j], xr[i]}, {R, R, W}, 0, 0);
    // L L^T d = r with the diagonal inverses: forward into D, backward into R
    for (int k = 0; k < T && rc == SPX_OK; ++k) {
      rc = ins(SPX_OP_TRMM, {V[k], xr[k], xd[k]}, {R, R, W}, 1, 0);
      for (int i = k + 1; i < T && rc == SPX_OK; ++i)
        rc = ins(SPX_OP_GEMM_FWD, {L.at(i, k), xd[k], xr[i]}, {R, R, W}, i == k + 1 ? 1 : 0, 0);
    }
    for (int k = T - 1; k >= 0 && rc == SPX_OK; --k) {
      rc = ins(SPX_OP_TRMM, {V[k], xd[k], xr[k]}, {R, R, W}, 1, 1);
      for (int i = k - 1; i >= 0 && rc == SPX_OK; --i)
        rc = ins(SPX_OP_GEMM_BWD, {L.at(k, i), xr[k], xd[i]}, {R, R, W}, i == k - 1 ? 1 : 0, 0);
    }
    // x += d
    for (int i = 0; i < T && rc == SPX_OK; ++i) rc = ins(SPX_OP_AXPY, {xr[i], xx[i]}, {R, W}, 0, 0);
  }
  if (out_ntasks) *out_ntasks = count;
  return rc;
}

extern "C" int spx_gemm_insert(spx_graph_t g, double* dev_A, double* dev_B, double* dev_C, int n,
                               int ld, int b, int commutative, long long* out_ntasks) {
  if (!g || !dev_A || !dev_B || !dev_C || n < 1 || b < 1 || ld < n || commutative < 0 ||
      commutative > 2)
    return SPX_ERR_INVALID_ARG;
  Tiles A, B, C;
  int rc = register_tiles(g, dev_A, n, n, ld, b, false, A);
  if (rc == SPX_OK) rc = register_tiles(g, dev_B, n, n, ld, b, false, B);
  if (rc == SPX_OK) rc = register_tiles(g, dev_C, n, n, ld, b, false, C);
  const int T = A.T;
  const int mode = commutative == 2   ? SPX_ATOMIC_WRITE
                   : commutative == 1 ? SPX_COMMUTATIVE_WRITE
                                      : SPX_WRITE;
  long long count = 0;
  for (int i = 0; i < T && rc == SPX_OK; ++i)
    for (int j = 0; j < T && rc == SPX_OK; ++j)
      for (int k = 0; k < T && rc == SPX_OK; ++k) {
        const unsigned hs[3] = {A.at(i, k), B.at(k, j), C.at(i, j)};
        const int ms[3] = {SPX_READ, SPX_READ, mode};
        rc = spx_task_insert(g, SPX_OP_GEMM_NN_ADD, hs, ms, 3, 0, SPX_F64, nullptr);
        if (rc == SPX_OK) ++count;
      }
  if (out_ntasks) *out_ntasks = count;
  return rc;
}

extern "C" int spx_gemm_insert_ozaki(spx_graph_t g, double* dev_A, double* dev_B, double* dev_C,
                                     int n, int ld, int b, int commutative, void* dev_S,
                                     long long S_bytes, long long* out_ntasks) {
  if (!g || !dev_A || !dev_B || !dev_C || n < 1 || ld < n || commutative < 0 ||
      commutative > 1 || !dev_S || ((uintptr_t)dev_S & 255))
    return SPX_ERR_INVALID_ARG;
  const long long slot = spx_ozaki_slot_bytes(b);
  if (!slot) return SPX_ERR_INVALID_ARG;
  const int T = (n + b - 1) / b;
  const long long nslots = 2LL * T * T;
  if (S_bytes < nslots * slot || nslots > 0x7FFFFFFF) return SPX_ERR_INVALID_ARG;
  int rc = spx_ozaki_register(g, dev_S, (int)nslots, b, nullptr);
  if (rc != SPX_OK) return rc;
  // A_ik owns slot i T + k, B_kj slot T^2 + k T + j
  Tiles A, B, C;
  A.T = B.T = T;
  A.b = B.b = b;
  A.h.assign((size_t)T * T, 0);
  B.h.assign((size_t)T * T, 0);
  char* S = (char*)dev_S;
  for (int i = 0; i < T && rc == SPX_OK; ++i)
    for (int j = 0; j < T && rc == SPX_OK; ++j) {
      const int r = n - i * b < b ? n - i * b : b;
      const int c = n - j * b < b ? n - j * b : b;
      const size_t off = (size_t)i * b * ld + (size_t)j * b;
      rc = spx_tile_register(g, dev_A + off, r, c, ld, SPX_DT_F64,
                             S + ((long long)i * T + j) * slot, b, &A.at(i, j));
      if (rc == SPX_OK)
        rc = spx_tile_register(g, dev_B + off, r, c, ld, SPX_DT_F64,
                               S + ((long long)T * T + (long long)i * T + j) * slot, b,
                               &B.at(i, j));
    }
  if (rc == SPX_OK) rc = register_tiles(g, dev_C, n, n, ld, b, false, C);
  long long count = 0;
  auto ins = [&](int op, std::initializer_list<unsigned> hs, std::initializer_list<int> ms) {
    const int r = spx_task_insert(g, op, hs.begin(), ms.begin(), (int)hs.size(), 0,
                                  SPX_F64_OZAKI, nullptr);
    if (r == SPX_OK) ++count;
    return r;
  };
  for (int i = 0; i < T && rc == SPX_OK; ++i)
    for (int k = 0; k < T && rc == SPX_OK; ++k) rc = ins(SPX_OP_SPLIT, {A.at(i, k)}, {SPX_WRITE});
  for (int k = 0; k < T && rc == SPX_OK; ++k)
    for (int j = 0; j < T && rc == SPX_OK; ++j) rc = ins(SPX_OP_SPLIT_T, {B.at(k, j)}, {SPX_WRITE});
  const int mode = commutative ? SPX_COMMUTATIVE_WRITE : SPX_WRITE;
  for (int i = 0; i < T && rc == SPX_OK; ++i)
    for (int j = 0; j < T && rc == SPX_OK; ++j)
      for (int k = 0; k < T && rc == SPX_OK; ++k)
        rc = ins(SPX_OP_GEMM_NN_ADD, {A.at(i, k), B.at(k, j), C.at(i, j)},
                 {SPX_READ, SPX_READ, mode});
  if (out_ntasks) *out_ntasks = count;
  return rc;
}

extern "C" int spx_axpy_insert(spx_graph_t g, float* dev_x, float* dev_y, long long n,
                               long long piece, double alpha, long long* out_ntasks) {
  if (!g || !dev_x || !dev_y || n < 1 || piece < 1 || dev_x == dev_y) return SPX_ERR_INVALID_ARG;
  long long count = 0;
  int rc = SPX_OK;
  for (long long p0 = 0; p0 < n && rc == SPX_OK; p0 += piece) {
    const long long len = n - p0 < piece ? n - p0 : piece;
    // a piece is a (len / 1024) x 1024 tile when 1024 divides it (so that its
    // 64-row units spread over CTAs), else one row
    const int cols = len % 1024 == 0 ? 1024 : (int)len;
    const long long rows = len / cols;
    if (rows > 0x7FFFFFFF || (len % 1024 != 0 && len > 0x7FFFFFFF)) return SPX_ERR_INVALID_ARG;
    unsigned hx = 0, hy = 0, id = 0;
    rc = spx_tile_register(g, dev_x + p0, (int)rows, cols, cols, SPX_DT_F32, nullptr, 0, &hx);
    if (rc == SPX_OK)
      rc = spx_tile_register(g, dev_y + p0, (int)rows, cols, cols, SPX_DT_F32, nullptr, 0, &hy);
    const unsigned hs[2] = {hx, hy};
    const int ms[2] = {SPX_READ, SPX_WRITE};
    if (rc == SPX_OK) rc = spx_task_insert(g, SPX_OP_AXPY, hs, ms, 2, 0, SPX_F64, &id);
    if (rc == SPX_OK && alpha != 1.0) rc = spx_task_set_scalar(g, id, alpha);
    if (rc == SPX_OK) ++count;
  }
  if (out_ntasks) *out_ntasks = count;
  return rc;
}

extern "C" int spx_nbody_insert(spx_graph_t g, int ngroups, double* const* dev_groups,
                                const int* sizes, int commutative, long long* out_ntasks) {
  if (!g || ngroups < 1 || !dev_groups || !sizes) return SPX_ERR_INVALID_ARG;
  std::vector<unsigned> h(ngroups);
  int rc = SPX_OK;
  for (int i = 0; i < ngroups && rc == SPX_OK; ++i) {
    if (!dev_groups[i] || sizes[i] < 1) return SPX_ERR_INVALID_ARG;
    rc = spx_tile_register(g, dev_groups[i], sizes[i], 8, 8, SPX_DT_F64, nullptr, 0, &h[i]);
  }
  const int W = commutative ? SPX_COMMUTATIVE_WRITE : SPX_WRITE;
  long long count = 0;
  for (int i = 0; i < ngroups && rc == SPX_OK; ++i) {
    const int m1[1] = {W};
    rc = spx_task_insert(g, SPX_OP_NBODY_SELF, &h[i], m1, 1, 0, SPX_F64, nullptr);
    if (rc == SPX_OK) ++count;
    for (int j = i + 1; j < ngroups && rc == SPX_OK; ++j) {
      const unsigned hs[2] = {h[i], h[j]};
      const int m2[2] = {W, W};
      rc = spx_task_insert(g, SPX_OP_NBODY_PAIR, hs, m2, 2, 0, SPX_F64, nullptr);
      if (rc == SPX_OK) ++count;
    }
  }
  if (out_ntasks) *out_ntasks = count;
  return rc;
}

extern "C" int spx_cholesky_insert_batch(spx_graph_t g, int count, double* const* dev_A,
                                         const int* n, const int* lda, const int* b,
                                         double* const* dev_X, const int* nrhs, const int* ldx,
                                         int lookahead, int prec, long long* out_ntasks) {
  if (!g || count < 0 || (count > 0 && (!dev_A || !n || !lda || !b))) return SPX_ERR_INVALID_ARG;
  long long total = 0;
  int rc = SPX_OK;
  for (int i = 0; i < count && rc == SPX_OK; ++i) {
    long long nt = 0;
    double* x = dev_X ? dev_X[i] : nullptr;
    rc = spx_cholesky_insert(g, dev_A[i], n[i], lda[i], b[i], x, x ? nrhs[i] : 0, x ? ldx[i] : 0,
                             lookahead, prec, &nt);
    total += nt;
  }
  if (out_ntasks) *out_ntasks = total;
  return rc;
}

extern "C" int spx_refine_insert(spx_graph_t g, double* dev_A0, int n, int lda, double* dev_L,
                                 int ldl, int b, double* dev_B, double* dev_X, double* dev_R,
                                 int nrhs, int ldx, int sweeps, long long* out_ntasks) {
  if (!g || !dev_A0 || !dev_L || !dev_B || !dev_X || !dev_R || n < 1 || b < 1 || lda < n ||
      ldl < n || nrhs < 1 || ldx < nrhs || sweeps < 0)
    return SPX_ERR_INVALID_ARG;
  Tiles A0, L;
  int rc = register_tiles(g, dev_A0, n, n, lda, b, false, A0);
  if (rc == SPX_OK) rc = register_tiles(g, dev_L, n, n, ldl, b, true, L);
  if (rc != SPX_OK) return rc;
  const int T = A0.T;
  std::vector<unsigned> xb(T), xx(T), xr(T);
  for (int i = 0; i < T && rc == SPX_OK; ++i) {
    const int r = n - i * b < b ? n - i * b : b;
    const size_t off = (size_t)i * b * ldx;
    rc = spx_tile_register(g, dev_B + off, r, nrhs, ldx, SPX_DT_F64, nullptr, 0, &xb[i]);
    if (rc == SPX_OK) rc = spx_tile_register(g, dev_X + off, r, nrhs, ldx, SPX_DT_F64, nullptr, 0, &xx[i]);
    if (rc == SPX_OK) rc = spx_tile_register(g, dev_R + off, r, nrhs, ldx, SPX_DT_F64, nullptr, 0, &xr[i]);
  }
  const int R = SPX_READ, W = SPX_WRITE;
  long long count = 0;
  auto ins = [&](int op, std::initializer_list<unsigned> hs, std::initializer_list<int> ms, int prio) {
    int r = spx_task_insert(g, op, hs.begin(), ms.begin(), (int)hs.size(), prio, SPX_F64, nullptr);
    if (r == SPX_OK) ++count;
    return r;
  };
  for (int sw = 0; sw < sweeps && rc == SPX_OK; ++sw) {
    // r = b - A0 x
    for (int i = 0; i < T && rc == SPX_OK; ++i) rc = ins(SPX_OP_COPY, {xb[i], xr[i]}, {R, W}, 0);
    for (int i = 0; i < T && rc == SPX_OK; ++i)
      for (int j = 0; j < T && rc == SPX_OK; ++j)
        rc = ins(SPX_OP_GEMM_FWD, {A0.at(i, j), xx[j], xr[i]}, {R, R, W}, 0);
    // L L^T d = r, d over r
    for (int k = 0; k < T && rc == SPX_OK; ++k) {
      rc = ins(SPX_OP_TRSM_L_FWD, {L.at(k, k), xr[k]}, {R, W}, 1);
      for (int i = k + 1; i < T && rc == SPX_OK; ++i)
        rc = ins(SPX_OP_GEMM_FWD, {L.at(i, k), xr[k], xr[i]}, {R, R, W}, i == k + 1 ? 1 : 0);
    }
    for (int k = T - 1; k >= 0 && rc == SPX_OK; --k) {
      rc = ins(SPX_OP_TRSM_LT_BWD, {L.at(k, k), xr[k]}, {R, W}, 1);
      for (int i = k - 1; i >= 0 && rc == SPX_OK; --i)
        rc = ins(SPX_OP_GEMM_BWD, {L.at(k, i), xr[k], xr[i]}, {R, R, W}, i == k - 1 ? 1 : 0);
    }
    // x += d
    for (int i = 0; i < T && rc == SPX_OK; ++i) rc = ins(SPX_OP_AXPY, {xr[i], xx[i]}, {R, W}, 0);
  }
  if (out_ntasks) *out_ntasks = count;
  return rc;
}
