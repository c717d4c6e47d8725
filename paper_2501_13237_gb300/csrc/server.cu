// Serving loop: whole extrapolation jobs (circuit, noise levels, observables,
// target lambda*) queued by nne_submit and run by worker threads, each with
// its own non-blocking stream and context, so that several jobs share the GPU
// at once (continuous batching).  Admission is first-in first-out and gated
// by the device-memory budget: the head job starts only when its bytes
// (nne_job_bytes, computed from the same allocation plan as nne_create_state)
// fit in what the running jobs leave free.
//
// Every job runs through the public entry points (nne_create_state,
// nne_build_superops, nne_apply_layer, nne_expect, nne_extrapolate); this
// file holds no arithmetic of the method.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// Deep copy of a job (nne_submit returns before the job runs).
struct JobCopy {
  uint64_t ticket = 0;
  int n = 0, n_layers = 0, n_lambda = 0, chi = 0, dtype = 0, trunc = 0;
  int sketch_rows = 0, sketch_cols = 0, power_iters = 0;
  int n_obs = 0, fit_method = 0, fit_degree = 0;
  double lambda_star = 1.0;
  bool has_bits = false;
  std::vector<int> layer_gates, layer_dir, left_qubit;
  std::vector<double> U, lambdas, rates, pauli;   // pauli: 32 per gate (c0, c1), empty for rate channels
  std::vector<char> sketch;
  std::vector<uint8_t> bits, paulis;
  size_t bytes = 0;
  long long gates = 0;
  int max_layer_gates = 0;
};

struct ResultRec {
  bool done = false;
  nne_status status = NNE_OK;
  std::string error;
  int n_lambda = 0, n_obs = 0;
  std::vector<double> values, log_fid, estimate;
  std::vector<int32_t> fit_status;
  double t_submit = 0, t_start = 0, t_end = 0;
  long long gate_steps = 0;
  size_t bytes = 0;
};

size_t r256(size_t b) { return ((b == 0 ? 16 : b) + 255) & ~size_t(255); }

}  // namespace

struct nne_server {
  int device = 0;
  int flags = 0;
  int dry_us = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<JobCopy>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<ResultRec>> results;
  size_t reserved = 0;
  int running = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::vector<std::thread> workers;
  FILE* log = nullptr;   // JSON-lines record of finished jobs (nne_server_set_log), guarded by mu
  std::unordered_map<uint64_t, nne_status> injected;   // nne_server_inject_failure, guarded by mu
  Clock::time_point t0 = Clock::now();
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// One JSON line per finished job (called with the server mutex held).
void log_job(FILE* f, const JobCopy& j, const ResultRec& r) {
  std::string err;
  for (char c : r.error) {
    if (c == '"' || c == '\\') err += '\\';
    if (static_cast<unsigned char>(c) >= 0x20) err += c;
  }
  std::fprintf(f,
               "{\"ticket\": %llu, \"status\": %d, \"error\": \"%s\", \"n\": %d, \"chi\": %d, "
               "\"n_lambda\": %d, \"gates\": %lld, \"gate_steps\": %lld, \"bytes\": %zu, "
               "\"t_submit\": %.6f, \"t_start\": %.6f, \"t_end\": %.6f, \"latency_s\": %.6f, \"log_fid\": [",
               (unsigned long long)j.ticket, (int)r.status, err.c_str(), j.n, j.chi, j.n_lambda, j.gates,
               r.gate_steps, r.bytes, r.t_submit, r.t_start, r.t_end, r.t_end - r.t_submit);
  for (size_t i = 0; i < r.log_fid.size(); ++i) {
    if (std::isfinite(r.log_fid[i]))
      std::fprintf(f, "%s%.17g", i ? ", " : "", r.log_fid[i]);
    else
      std::fprintf(f, "%snull", i ? ", " : "");
  }
  std::fprintf(f, "]}\n");
  std::fflush(f);
}

nne_status run_job(nne_ctx* ctx, cudaStream_t st, const JobCopy& j, ResultRec& r) {
  nne_state* s = nullptr;
  nne_status rc = nne_create_state(ctx, j.n, j.chi, j.n_lambda, (nne_dtype)j.dtype, (nne_trunc)j.trunc,
                                   j.has_bits ? j.bits.data() : nullptr, &s);
  if (rc != NNE_OK) return rc;
  double* dU = nullptr;
  double* dRates = nullptr;
  double* dG = nullptr;
  auto cleanup = [&]() {
    if (dU) cudaFreeAsync(dU, st);
    if (dRates) cudaFreeAsync(dRates, st);
    if (dG) cudaFreeAsync(dG, st);
    nne_destroy_state(s);
  };
  if (j.trunc == NNE_TRUNC_RSVD) {
    rc = nne_set_sketch(s, j.sketch.data(), j.sketch_rows, j.sketch_cols, j.power_iters);
    if (rc != NNE_OK) {
      cleanup();
      return rc;
    }
  }
  // rate channels: dRates = n_lambda x 4; Pauli channels: 32 per gate (c0, c1), then the n_lambda levels
  const bool pauli = !j.pauli.empty();
  const size_t n_rates = pauli ? (size_t)32 * j.gates + j.n_lambda : (size_t)4 * j.n_lambda;
  cudaError_t e = cudaMallocAsync((void**)&dU, sizeof(double) * 32 * (size_t)std::max<long long>(j.gates, 1), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&dRates, sizeof(double) * n_rates, st);
  if (e == cudaSuccess)
    e = cudaMallocAsync((void**)&dG, sizeof(double) * 512 * (size_t)j.n_lambda * std::max(j.max_layer_gates, 1), st);
  if (e == cudaSuccess && j.gates > 0)
    e = cudaMemcpyAsync(dU, j.U.data(), sizeof(double) * 32 * j.gates, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !pauli)
    e = cudaMemcpyAsync(dRates, j.rates.data(), sizeof(double) * 4 * j.n_lambda, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && pauli)
    e = cudaMemcpyAsync(dRates, j.pauli.data(), sizeof(double) * 32 * j.gates, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && pauli)
    e = cudaMemcpyAsync(dRates + 32 * j.gates, j.lambdas.data(), sizeof(double) * j.n_lambda, cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host vectors are the job's own; keep them simple
  if (e != cudaSuccess) {
    cleanup();
    return nne::set_cuda_error(e, "server staging", __FILE__, __LINE__);
  }
  long long off = 0;
  for (int l = 0; l < j.n_layers && rc == NNE_OK; ++l) {
    const int g = j.layer_gates[l];
    if (g == 0) continue;
    rc = pauli ? nne_build_pauli_superops(ctx, g, dU + 32 * off, dRates + 32 * off, j.n_lambda, dRates + 32 * j.gates,
                                          dG)
               : nne_build_superops(ctx, g, dU + 32 * off, j.n_lambda, dRates, dG);
    if (rc == NNE_OK) rc = nne_apply_layer(s, g, j.left_qubit.data() + off, dG, j.layer_dir[l]);
    off += g;
  }
  if (rc == NNE_OK) {
    std::vector<double> re((size_t)j.n_lambda * std::max(j.n_obs, 1)), im(re.size());
    r.log_fid.assign(j.n_lambda, 0.0);
    rc = nne_expect(s, j.n_obs, j.paulis.data(), re.data(), im.data(), r.log_fid.data());
    if (rc == NNE_OK) {
      r.values.assign(re.begin(), re.begin() + (size_t)j.n_lambda * j.n_obs);
      r.estimate.assign(j.n_obs, 0.0);
      r.fit_status.assign(j.n_obs, 0);
      if (j.n_obs > 0)
        rc = nne_extrapolate(ctx, j.n_lambda, j.lambdas.data(), r.values.data(), r.log_fid.data(), j.n_obs,
                             j.fit_method, j.fit_degree, j.lambda_star, nullptr, r.estimate.data(),
                             r.fit_status.data());
    }
  }
  r.gate_steps = j.gates * j.n_lambda;
  cleanup();
  cudaStreamSynchronize(st);
  return rc;
}

void worker_main(nne_server* srv) {
  const bool dry = (srv->flags & NNE_SERVER_DRYRUN) != 0;
  cudaStream_t st = nullptr;
  nne_ctx* ctx = nullptr;
  nne_status init_rc = NNE_OK;
  std::string init_err;
  if (!dry) {
    if (cudaSetDevice(srv->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      init_rc = NNE_ERR_CUDA;
      init_err = "worker could not create its stream";
    } else if ((init_rc = nne_ctx_create(srv->device, st, 0, &ctx)) != NNE_OK) {
      init_err = nne_last_error();
    }
  }
  nne_status injected_rc = NNE_OK;
  for (;;) {
    std::shared_ptr<JobCopy> job;
    std::shared_ptr<ResultRec> res;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      srv->cv_work.wait(lk, [&] {
        return srv->stop ||
               (!srv->queue.empty() && (srv->budget == 0 || srv->reserved + srv->queue.front()->bytes <= srv->budget));
      });
      if (srv->stop) break;
      job = srv->queue.front();
      srv->queue.pop_front();
      srv->reserved += job->bytes;
      srv->running++;
      res = srv->results[job->ticket];
      res->t_start = srv->now();
      res->bytes = job->bytes;
      auto inj = srv->injected.find(job->ticket);
      if (inj != srv->injected.end()) {
        injected_rc = inj->second;
        srv->injected.erase(inj);
      }
    }
    nne_status rc;
    std::string err;
    if (injected_rc != NNE_OK) {
      rc = injected_rc;
      err = "injected failure";
      injected_rc = NNE_OK;
    } else if (dry) {
      std::this_thread::sleep_for(std::chrono::microseconds(srv->dry_us));
      rc = NNE_ERR_UNIMPL;
      err = "dry run: no GPU work";
    } else if (init_rc != NNE_OK) {
      rc = init_rc;
      err = init_err;
    } else {
      rc = run_job(ctx, st, *job, *res);
      if (rc != NNE_OK) err = nne_last_error();
    }
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      res->status = rc;
      res->error = err;
      res->t_end = srv->now();
      res->done = true;
      if (srv->log) log_job(srv->log, *job, *res);
      srv->reserved -= job->bytes;
      srv->running--;
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
  if (ctx) nne_ctx_destroy(ctx);
  if (st) cudaStreamDestroy(st);
}

nne_status copy_job(const nne_job* j, JobCopy& c) {
  if (!j || j->n_qubits < 2 || j->n_layers < 0 || (j->n_layers > 0 && (!j->layer_gates || !j->layer_dir)) ||
      j->n_lambda < 1 || j->n_lambda > 64 || !j->lambdas || (!j->rates && !j->pauli_rates) || j->chi < 1 ||
      j->chi > 4096 ||
      (j->dtype != NNE_C64 && j->dtype != NNE_C128) || (j->trunc != NNE_TRUNC_EXACT && j->trunc != NNE_TRUNC_RSVD) ||
      j->n_obs < 0 || (j->n_obs > 0 && !j->paulis) || j->fit_method < 0 || j->fit_method > 2 ||
      (j->fit_method == NNE_FIT_POLY && (j->fit_degree < 1 || j->fit_degree > 15)))
    return nne::set_error(NNE_ERR_ARG, "nne_submit: bad job");
  c.n = j->n_qubits;
  c.n_layers = j->n_layers;
  c.n_lambda = j->n_lambda;
  c.chi = j->chi;
  c.dtype = j->dtype;
  c.trunc = j->trunc;
  c.n_obs = j->n_obs;
  c.fit_method = j->fit_method;
  c.fit_degree = j->fit_degree;
  c.lambda_star = j->lambda_star;
  c.layer_gates.assign(j->layer_gates, j->layer_gates + j->n_layers);
  c.layer_dir.assign(j->layer_dir, j->layer_dir + j->n_layers);
  long long gates = 0;
  for (int l = 0; l < c.n_layers; ++l) {
    if (c.layer_gates[l] < 0 || (c.layer_dir[l] != 1 && c.layer_dir[l] != -1))
      return nne::set_error(NNE_ERR_ARG, "nne_submit: layer %d: bad gate count or direction", l);
    gates += c.layer_gates[l];
    c.max_layer_gates = std::max(c.max_layer_gates, c.layer_gates[l]);
  }
  c.gates = gates;
  if (gates > 0 && (!j->left_qubit || !j->U)) return nne::set_error(NNE_ERR_ARG, "nne_submit: gates without data");
  c.left_qubit.assign(j->left_qubit, j->left_qubit + gates);
  for (long long g = 0; g < gates; ++g)
    if (c.left_qubit[g] < 0 || c.left_qubit[g] > c.n - 2)
      return nne::set_error(NNE_ERR_ARG, "nne_submit: gate %lld: left qubit %d out of range", g, c.left_qubit[g]);
  c.U.assign(j->U, j->U + 32 * gates);
  c.lambdas.assign(j->lambdas, j->lambdas + c.n_lambda);
  if (j->pauli_rates) {
    c.pauli.assign(j->pauli_rates, j->pauli_rates + 32 * gates);
    for (long long g = 0; g < gates; ++g)
      for (int i = 0; i < c.n_lambda; ++i) {
        double tot = 0;
        for (int ab = 0; ab < 16; ++ab) {
          const double p = c.pauli[32 * g + ab] + c.lambdas[i] * c.pauli[32 * g + 16 + ab];
          if (!(p >= -1e-12 && p <= 1.0 + 1e-12))
            return nne::set_error(NNE_ERR_ARG, "nne_submit: gate %lld level %d: Pauli probability %g", g, i, p);
          tot += p;
        }
        if (!(std::fabs(tot - 1.0) <= 1e-12))
          return nne::set_error(NNE_ERR_ARG, "nne_submit: gate %lld level %d: Pauli probabilities sum to %.17g", g,
                                i, tot);
      }
  } else {
    c.rates.assign(j->rates, j->rates + 4 * c.n_lambda);
    for (int i = 0; i < c.n_lambda; ++i)
      for (int k = 0; k < 4; ++k) {
        const double p = c.rates[4 * i + k];
        if (!(p >= 0.0 && p <= (k == 0 ? 16.0 / 15.0 : 1.0)))
          return nne::set_error(NNE_ERR_ARG, "nne_submit: rate %d of level %d out of range: %g", k, i, p);
      }
  }
  if (c.trunc == NNE_TRUNC_RSVD) {
    if (!j->sketch || j->sketch_rows < 1 || j->sketch_cols < 1 || j->power_iters < 0)
      return nne::set_error(NNE_ERR_ARG, "nne_submit: randomized truncation needs a sketch");
    c.sketch_rows = j->sketch_rows;
    c.sketch_cols = j->sketch_cols;
    c.power_iters = j->power_iters;
    const size_t b = (size_t)c.sketch_rows * c.sketch_cols * (c.dtype == NNE_C64 ? 8 : 16);
    c.sketch.assign((const char*)j->sketch, (const char*)j->sketch + b);
  }
  c.has_bits = j->init_bits != nullptr;
  if (c.has_bits) c.bits.assign(j->init_bits, j->init_bits + c.n);
  c.paulis.assign(j->paulis, j->paulis + (size_t)c.n_obs * c.n);
  for (uint8_t p : c.paulis)
    if (p > 3) return nne::set_error(NNE_ERR_ARG, "nne_submit: Pauli code %d", (int)p);
  c.bytes = nne_job_bytes(j);
  return NNE_OK;
}

}  // namespace

extern "C" {

size_t nne_job_bytes(const nne_job* j) {
  if (!j || j->n_qubits < 2 || j->chi < 1 || j->n_lambda < 1) return 0;
  long long gates = 0;
  int maxg = 0;
  for (int l = 0; l < j->n_layers; ++l) {
    gates += j->layer_gates[l];
    maxg = std::max(maxg, j->layer_gates[l]);
  }
  const int sk_cols = j->trunc == NNE_TRUNC_RSVD ? j->sketch_cols : 0;
  size_t b = nne::state_bytes(j->n_qubits, j->chi, j->n_lambda, j->dtype, j->sketch_rows, sk_cols);
  // staged gates, rates and one layer of superoperators (run_job)
  const size_t n_rates = j->pauli_rates ? (size_t)32 * gates + j->n_lambda : (size_t)4 * j->n_lambda;
  b += r256(sizeof(double) * 32 * (size_t)std::max<long long>(gates, 1)) + r256(sizeof(double) * n_rates) +
       r256(sizeof(double) * 512 * (size_t)j->n_lambda * std::max(maxg, 1));
  // superoperator-build scratch of the worker's context, expectation and fit temporaries
  const size_t no = (size_t)std::max(j->n_obs, 1);
  b += r256(sizeof(double) * 512 * j->n_lambda) + r256(no * j->n_qubits) + 2 * r256(sizeof(int) * no) +
       r256(sizeof(double) * 2 * no * j->n_lambda) + 3 * r256(sizeof(double) * j->n_lambda) +
       3 * r256(sizeof(double) * no) + r256(sizeof(double) * no * j->n_lambda);
  return b;
}

nne_status nne_server_create(int device, size_t hbm_budget_bytes, int n_workers, int flags, int dry_run_us,
                             nne_server** out) {
  if (!out || n_workers < 1 || n_workers > 64 || dry_run_us < 0)
    return nne::set_error(NNE_ERR_ARG, "nne_server_create: bad arguments");
  *out = nullptr;
  if (!(flags & NNE_SERVER_DRYRUN)) {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return nne::set_cuda_error(e, "cudaGetDeviceCount", __FILE__, __LINE__);
    if (device < 0 || device >= ndev) return nne::set_error(NNE_ERR_ARG, "device %d out of range", device);
  }
  nne_server* s = new nne_server();
  s->device = device;
  s->flags = flags;
  s->dry_us = dry_run_us;
  s->budget = hbm_budget_bytes;
  for (int i = 0; i < n_workers; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return NNE_OK;
}

nne_status nne_submit(nne_server* srv, const nne_job* job, uint64_t* ticket) {
  if (!srv || !ticket) return nne::set_error(NNE_ERR_ARG, "nne_submit: bad arguments");
  auto c = std::make_shared<JobCopy>();
  nne_status rc = copy_job(job, *c);
  if (rc != NNE_OK) return rc;
  if (srv->budget && c->bytes > srv->budget)
    return nne::set_error(NNE_ERR_OOM, "nne_submit: job needs %zu bytes, budget is %zu", c->bytes, srv->budget);
  auto r = std::make_shared<ResultRec>();
  r->n_lambda = c->n_lambda;
  r->n_obs = c->n_obs;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return nne::set_error(NNE_ERR_ARG, "nne_submit: server is shutting down");
    c->ticket = srv->next_ticket++;
    r->t_submit = srv->now();
    srv->results[c->ticket] = r;
    srv->queue.push_back(c);
    *ticket = c->ticket;
  }
  srv->cv_work.notify_all();
  return NNE_OK;
}

nne_status nne_poll(nne_server* srv, uint64_t ticket, int timeout_ms, nne_result* out) {
  if (!srv || !out) return nne::set_error(NNE_ERR_ARG, "nne_poll: bad arguments");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->results.find(ticket);
  if (it == srv->results.end()) return nne::set_error(NNE_ERR_ARG, "nne_poll: unknown ticket %llu",
                                                      (unsigned long long)ticket);
  std::shared_ptr<ResultRec> r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_ms < 0) srv->cv_done.wait(lk, ready);
  else if (timeout_ms > 0) srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  if (!r->done) return NNE_PENDING;
  out->status = r->status;
  std::snprintf(out->error, sizeof(out->error), "%s", r->error.c_str());
  if (out->values && !r->values.empty()) std::memcpy(out->values, r->values.data(), sizeof(double) * r->values.size());
  if (out->log_fid && !r->log_fid.empty())
    std::memcpy(out->log_fid, r->log_fid.data(), sizeof(double) * r->log_fid.size());
  if (out->estimate && !r->estimate.empty())
    std::memcpy(out->estimate, r->estimate.data(), sizeof(double) * r->estimate.size());
  if (out->fit_status && !r->fit_status.empty())
    std::memcpy(out->fit_status, r->fit_status.data(), sizeof(int32_t) * r->fit_status.size());
  out->t_submit = r->t_submit;
  out->t_start = r->t_start;
  out->t_end = r->t_end;
  out->gate_steps = r->gate_steps;
  out->bytes_reserved = r->bytes;
  srv->results.erase(it);
  return NNE_OK;
}

nne_status nne_server_inject_failure(nne_server* srv, uint64_t ticket, nne_status status) {
  if (!srv || status >= 0) return nne::set_error(NNE_ERR_ARG, "nne_server_inject_failure: bad arguments");
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->results.find(ticket);
  if (it == srv->results.end() || it->second->done || it->second->t_start > 0)
    return nne::set_error(NNE_ERR_ARG, "nne_server_inject_failure: ticket %llu is not waiting",
                          (unsigned long long)ticket);
  srv->injected[ticket] = status;
  return NNE_OK;
}

nne_status nne_cancel(nne_server* srv, uint64_t ticket) {
  if (!srv) return nne::set_error(NNE_ERR_ARG, "nne_cancel: null server");
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->results.find(ticket);
    if (it == srv->results.end() || it->second->done)
      return nne::set_error(NNE_ERR_ARG, "nne_cancel: unknown or finished ticket %llu", (unsigned long long)ticket);
    auto q = std::find_if(srv->queue.begin(), srv->queue.end(),
                          [&](const std::shared_ptr<JobCopy>& j) { return j->ticket == ticket; });
    if (q == srv->queue.end()) return NNE_PENDING;   // running: it completes normally
    std::shared_ptr<JobCopy> job = *q;
    srv->queue.erase(q);
    ResultRec& r = *it->second;
    r.status = NNE_ERR_CANCELLED;
    r.error = "cancelled before it started";
    r.t_start = r.t_end = srv->now();
    r.done = true;
    if (srv->log) log_job(srv->log, *job, r);
  }
  srv->cv_done.notify_all();
  srv->cv_work.notify_all();   // the queue head may have changed
  return NNE_OK;
}

void nne_server_stats(nne_server* srv, int* queued, int* running, int* done, size_t* bytes_reserved) {
  if (!srv) return;
  std::lock_guard<std::mutex> lk(srv->mu);
  int d = 0;
  for (auto& kv : srv->results) d += kv.second->done ? 1 : 0;
  if (queued) *queued = (int)srv->queue.size();
  if (running) *running = srv->running;
  if (done) *done = d;
  if (bytes_reserved) *bytes_reserved = srv->reserved;
}

void nne_server_destroy(nne_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->queue.clear();
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  if (srv->log) std::fclose(srv->log);
  delete srv;
}

nne_status nne_server_set_log(nne_server* srv, const char* path) {
  if (!srv) return nne::set_error(NNE_ERR_ARG, "nne_server_set_log: null server");
  FILE* f = nullptr;
  if (path && !(f = std::fopen(path, "a"))) return nne::set_error(NNE_ERR_ARG, "nne_server_set_log: cannot open %s", path);
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->log) std::fclose(srv->log);
  srv->log = f;
  return NNE_OK;
}

}  // extern "C"
