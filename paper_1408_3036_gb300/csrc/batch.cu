// Many independent cells on one GPU.
//
// The cells of a batch differ in grid, cutoff and occupied count, so their
// kernels are specialised to different geometries and cannot share launches.
// Small cells leave most of the 152 SMs idle when run one after another; here
// each cell gets its own context and its own non-blocking stream, and a pool of
// host workers drives the cells' Lanczos recursions concurrently so that the
// kernels of several cells fill the GPU together.  A context is used by one
// worker at a time (a worker takes a whole cell, all of its frequencies), and
// the cooperative CG launches of concurrent cells each take an equal share of
// the resident CTA slots, so all of them can be resident at once.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <string>
#include <thread>
#include <vector>

#include "gw.h"

void gw_internal_set_cta_div(gw_ctx* ctx, int n);

struct gw_batch {
  int dev = 0;
  int workers = 1;
  std::vector<gw_ctx*> cells;
  std::vector<cudaStream_t> streams;
  std::string err;
};

namespace {

constexpr int kMaxWorkers = 32;

void free_batch(gw_batch* b) {
  for (gw_ctx* c : b->cells)
    if (c) gw_destroy(c);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  delete b;
}

}  // namespace

extern "C" {

gw_status gw_batch_setup(gw_batch** out, int n_cells, const double* L, const int* n_grid, const double* ecut,
                         const double* const* vloc, int coulomb, int n_workers) {
  if (!out) return GW_E_ARG;
  *out = nullptr;
  if (n_cells < 1 || !L || !n_grid || !ecut || !vloc) return GW_E_ARG;
  gw_batch* b = new gw_batch();
  if (cudaGetDevice(&b->dev) != cudaSuccess) {
    delete b;
    return GW_E_CUDA;
  }
  b->workers = std::min(n_workers > 0 ? n_workers : 8, std::min(n_cells, kMaxWorkers));
  b->cells.assign(n_cells, nullptr);
  b->streams.assign(n_cells, nullptr);
  for (int i = 0; i < n_cells; ++i) {
    if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      free_batch(b);
      return GW_E_CUDA;
    }
    gw_status st = gw_setup(&b->cells[i], L[i], n_grid[i], ecut[i], vloc[i], coulomb, b->streams[i]);
    if (st != GW_OK) {
      free_batch(b);
      return st;
    }
    gw_internal_set_cta_div(b->cells[i], b->workers);
  }
  *out = b;
  return GW_OK;
}

int gw_batch_size(const gw_batch* b) { return b ? (int)b->cells.size() : 0; }

gw_ctx* gw_batch_cell(gw_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->cells.size()) return nullptr;
  return b->cells[i];
}

gw_status gw_batch_lanczos(gw_batch* b, const double* const* start, int k, int n_omega, const double* omega,
                           double* alpha, double* beta, gw_prec prec, int* cell_status) {
  if (!b) return GW_E_ARG;
  const int n = (int)b->cells.size();
  if (!start || !omega || !alpha || !beta || k < 1 || n_omega < 1) {
    b->err = "gw_batch_lanczos: null pointer or non-positive k / n_omega";
    return GW_E_ARG;
  }
  for (int i = 0; i < n; ++i)
    if (!start[i]) {
      b->err = "gw_batch_lanczos: start[" + std::to_string(i) + "] is null";
      return GW_E_ARG;
    }
  // Largest cells first, so the long jobs do not start last.
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) cost[i] = (double)gw_npw(b->cells[i]);
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });

  std::vector<int> status(n, GW_OK);
  std::vector<std::string> msgs(n);
  std::atomic<int> next{0};
  const size_t ka = (size_t)n_omega * k, kb = (size_t)n_omega * (k > 1 ? k - 1 : 0);
  auto work = [&]() {
    if (cudaSetDevice(b->dev) != cudaSuccess) return;
    for (int j = next.fetch_add(1); j < n; j = next.fetch_add(1)) {
      const int i = order[j];
      gw_ctx* c = b->cells[i];
      std::vector<double> a(2 * (size_t)k), bb(2 * (size_t)std::max(k - 1, 1));
      for (int w = 0; w < n_omega; ++w) {
        double* ao = alpha + 2 * ((size_t)i * ka + (size_t)w * k);
        double* bo = beta + 2 * ((size_t)i * kb + (size_t)w * (k > 1 ? k - 1 : 0));
        gw_status st;
        const double* om = omega + 2 * ((size_t)i * n_omega + w);
        if (om[1] == 0.0) {
          // real frequency: Hermitian Lanczos, real alpha and beta
          st = gw_lanczos(c, start[i], 1, k, om, a.data(), bb.data(), nullptr, prec, 0);
          for (int m = 0; m < k; ++m) {
            ao[2 * m] = a[m];
            ao[2 * m + 1] = 0.0;
          }
          for (int m = 0; m + 1 < k; ++m) {
            bo[2 * m] = bb[m];
            bo[2 * m + 1] = 0.0;
          }
        } else {
          // complex frequency: complex-symmetric (bilinear) recursion, block size 1
          st = gw_block_lanczos(c, start[i], 1, k, om, a.data(), bb.data(), nullptr, prec, 0);
          std::copy(a.begin(), a.begin() + 2 * k, ao);
          if (k > 1) std::copy(bb.begin(), bb.begin() + 2 * (k - 1), bo);
        }
        if (st != GW_OK) {
          status[i] = st;
          msgs[i] = gw_last_error(c);
          break;
        }
      }
    }
  };
  std::vector<std::thread> pool;
  const int nw = std::min(b->workers, n);
  for (int t = 1; t < nw; ++t) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();

  gw_status first = GW_OK;
  b->err.clear();
  for (int i = 0; i < n; ++i) {
    if (cell_status) cell_status[i] = status[i];
    if (status[i] != GW_OK && first == GW_OK) {
      first = (gw_status)status[i];
      b->err = "cell " + std::to_string(i) + ": " + msgs[i];
    }
  }
  return first;
}

const char* gw_batch_last_error(const gw_batch* b) { return b ? b->err.c_str() : "null batch"; }

void gw_batch_destroy(gw_batch* b) {
  if (b) free_batch(b);
}

}  // extern "C"
