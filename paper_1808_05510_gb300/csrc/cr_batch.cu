// Batched lambda x fold sweep: many independent greedy solves (Algorithm 1)
// of sub-problems of one data set, run concurrently on one GPU.
//
// A single greedy solve is a chain of dependent steps whose PCG sub-solves
// each live on one thread-block cluster (16 of the 152 SMs), so one solve
// leaves most of the GPU idle.  The sweep keeps `concurrency` solves in
// flight: each worker thread owns a CUDA stream and takes the next member from
// a shared queue (largest lambda first: the sub-problems' conditioning, and so
// the PCG work, grows with lambda), builds its sub-problem (the member's
// injection columns of X, Y and Omega), runs cr_solve and scores the held-out
// columns with cr_cv_error.  The workers' streams fork from the caller's
// stream and join back into it.  Member problems are destroyed only after the
// last member finishes: a device free synchronises the whole device and would
// stall the other workers.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "conreg.h"
#include "cr_common.cuh"

namespace cr {
void set_global_error(const std::string& msg);
cr_status adopt_stream(cr_problem* p, cudaStream_t st);
}

namespace {

struct Worker {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  // host gather buffers for the member's columns
  std::vector<double> X, Y;
  std::vector<uint8_t> Om;
  std::vector<double> Xt, Yt;
  std::vector<uint8_t> Omt;
};

void gather(const double* src, int64_t ld, int64_t rows, const int32_t* cols, int32_t n, std::vector<double>& dst) {
  dst.resize((size_t)rows * std::max(n, 1));
  for (int32_t k = 0; k < n; ++k) std::memcpy(&dst[(size_t)k * rows], src + cols[k] * ld, sizeof(double) * rows);
}

void gather(const uint8_t* src, int64_t ld, int64_t rows, const int32_t* cols, int32_t n, std::vector<uint8_t>& dst) {
  dst.resize((size_t)rows * std::max(n, 1));
  for (int32_t k = 0; k < n; ++k) std::memcpy(&dst[(size_t)k * rows], src + cols[k] * ld, rows);
}

bool cols_ok(const int32_t* c, int32_t n, int64_t m) {
  if (n > 0 && !c) return false;
  for (int32_t k = 0; k < n; ++k)
    if (c[k] < 0 || c[k] >= m) return false;
  return true;
}

}  // namespace

extern "C" cr_status cr_solve_batch(const cr_problem_desc* desc_in, const cr_options* opts,
                                    const cr_member* members, int32_t n_members, int32_t r_max, double tau,
                                    double relres_target, int32_t concurrency, cr_member_result* results,
                                    cr_problem** keep) {
  if (!desc_in || !members || !results || n_members < 0 || r_max < 0 || !(tau >= 0.0)) {
    cr::set_global_error("cr_solve_batch: bad arguments");
    return CR_EINVAL;
  }
  // device inputs are staged once; every member gathers its columns from the host copy
  cr::DescCopy staged;
  cr_problem_desc dview;
  {
    std::string err;
    const cr_status ss = cr::stage_desc(desc_in, &staged, &dview, err);
    if (ss != CR_OK) {
      cr::set_global_error("cr_solve_batch: " + err);
      return ss;
    }
  }
  const cr_problem_desc* desc = &dview;
  for (int32_t k = 0; k < n_members; ++k) {
    const cr_member& mb = members[k];
    if (mb.n_fit < 1 || mb.n_test < 0 || !cols_ok(mb.fit_cols, mb.n_fit, desc->ninj) ||
        !cols_ok(mb.test_cols, mb.n_test, desc->ninj) || !(mb.lambda > 0.0)) {
      cr::set_global_error("cr_solve_batch: member " + std::to_string(k) + " has bad columns or lambda");
      return CR_EINVAL;
    }
  }
  std::memset(results, 0, sizeof(cr_member_result) * (size_t)n_members);
  if (keep) std::fill(keep, keep + n_members, nullptr);
  if (n_members == 0) return CR_OK;

  cr_options base{};
  if (opts) {
    base = *opts;
  } else {
    cr_options_default(&base);
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int S = concurrency > 0 ? concurrency : std::max(1, sms / 16);
  S = std::min(S, n_members);
  // share the persistent Galerkin kernel's CTAs between the members in flight
  if (base.galerkin_ctas <= 0 && S > 1) base.galerkin_ctas = std::max(1, sms / S);
  cudaStream_t caller = (cudaStream_t)base.stream;

  // longest first: order by lambda, descending (ties: given order)
  std::vector<int32_t> order(n_members);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return members[a].lambda > members[b].lambda; });

  std::vector<Worker> W(S);
  cudaEvent_t fork = nullptr;
  if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(fork, caller) != cudaSuccess) {
    cudaGetLastError();
    cr::set_global_error("cr_solve_batch: event creation failed");
    return CR_ECUDA;
  }
  for (auto& w : W) {
    if (cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamWaitEvent(w.st, fork, 0) != cudaSuccess) {
      cudaGetLastError();
      for (auto& x : W) {
        if (x.st) cudaStreamDestroy(x.st);
        if (x.done) cudaEventDestroy(x.done);
      }
      cudaEventDestroy(fork);
      cr::set_global_error("cr_solve_batch: stream creation failed");
      return CR_ECUDA;
    }
  }

  std::vector<cr_problem*> probs(n_members, nullptr);
  std::atomic<int32_t> next{0};
  auto run = [&](int slot) {
    cudaSetDevice(dev);
    Worker& w = W[slot];
    for (;;) {
      const int32_t q = next.fetch_add(1);
      if (q >= n_members) break;
      const int32_t k = order[q];
      const cr_member& mb = members[k];
      cr_member_result& res = results[k];
      res.slot = slot;
      const auto t0 = std::chrono::steady_clock::now();
      gather(desc->X_host, desc->ldx, desc->nx, mb.fit_cols, mb.n_fit, w.X);
      gather(desc->Y_host, desc->ldy, desc->ny, mb.fit_cols, mb.n_fit, w.Y);
      gather(desc->Omega_host, desc->ldo, desc->ny, mb.fit_cols, mb.n_fit, w.Om);
      cr_problem_desc d = *desc;
      d.ninj = mb.n_fit;
      d.X_host = w.X.data();
      d.ldx = desc->nx;
      d.Y_host = w.Y.data();
      d.ldy = desc->ny;
      d.Omega_host = w.Om.data();
      d.ldo = desc->ny;
      d.lambda = mb.lambda;
      cr_options o = base;
      o.stream = w.st;
      cr_problem* p = nullptr;
      cr_status s = cr_create(&d, &o, &p);
      if (s != CR_OK) {
        res.status = s;
        continue;
      }
      probs[k] = p;
      cr_solve_info si{};
      s = cr_solve(p, r_max, tau, relres_target, &si);
      res.status = s;
      res.rank = si.rank;
      res.stop = si.stop;
      res.relres = si.relres;
      res.dW = si.dW;
      res.J = si.J;
      res.pcg_iters = si.pcg_iters;
      res.cg_iters = si.cg_iters;
      if ((s == CR_OK || s == CR_ENOTCONV) && mb.n_test > 0) {
        gather(desc->X_host, desc->ldx, desc->nx, mb.test_cols, mb.n_test, w.Xt);
        gather(desc->Y_host, desc->ldy, desc->ny, mb.test_cols, mb.n_test, w.Yt);
        gather(desc->Omega_host, desc->ldo, desc->ny, mb.test_cols, mb.n_test, w.Omt);
        const cr_status sc = cr_cv_error(p, mb.n_test, w.Xt.data(), desc->nx, w.Yt.data(), desc->ny, w.Omt.data(),
                                         desc->ny, &res.cv_num, &res.cv_den);
        if (sc != CR_OK) res.status = sc;
      }
      res.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    cudaEventRecord(w.done, w.st);
  };
  std::vector<std::thread> threads;
  threads.reserve(S);
  for (int t = 0; t < S; ++t) threads.emplace_back(run, t);
  for (auto& t : threads) t.join();
  for (auto& w : W) cudaStreamWaitEvent(caller, w.done, 0);

  cr_status rc = CR_OK;
  for (int32_t k = 0; k < n_members && rc == CR_OK; ++k)
    if (results[k].status != CR_OK && results[k].status != CR_ENOTCONV) rc = (cr_status)results[k].status;
  if (keep) {
    // the workers' streams end with this call: kept problems move to the caller's stream
    for (auto* p : probs) {
      const cr_status s = p ? cr::adopt_stream(p, caller) : CR_OK;
      if (s != CR_OK && rc == CR_OK) rc = s;
    }
    std::copy(probs.begin(), probs.end(), keep);
  } else {
    for (auto* p : probs) cr_destroy(p);
  }
  for (auto& w : W) {
    cudaStreamSynchronize(w.st);
    cudaStreamDestroy(w.st);
    cudaEventDestroy(w.done);
  }
  cudaEventDestroy(fork);
  return rc;
}
