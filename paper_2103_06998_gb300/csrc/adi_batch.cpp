// Batched mode: many independent ADI problems stepped by one CUDA graph per
// step (see the batch section of include/adi_maxwell.h), and the line-tile
// autotuner.
#include <cuda_runtime.h>

#include <cstdio>
#include <fstream>
#include <map>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "adi_internal.h"

struct adi_batch_ctx {
  std::vector<adi_handle> inst;
  std::vector<cudaStream_t> streams;  // one per instance, used while capturing
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaStream_t stream = nullptr;      // the batch stream (own_stream or the caller's)
  cudaStream_t own_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::string err;
};

namespace {

adi_status bfail(adi_batch b, adi_status s, const std::string& m) {
  if (b) b->err = m;
  return adi::fail_global(s, m);
}

void drop_batch_graph(adi_batch b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

void free_batch(adi_batch b) {
  if (!b) return;
  drop_batch_graph(b);
  for (adi_handle h : b->inst) adi_destroy(h);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
}

// One step of every instance, each on its own stream, forked from and joined
// to the batch stream (run while the batch stream is being captured).
cudaError_t record_step(adi_batch b) {
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (size_t i = 0; i < b->inst.size() && e == cudaSuccess; ++i) {
    adi::Ctx& c = *b->inst[i];
    cudaStream_t own = c.stream;
    e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
    c.stream = b->streams[i];
    if (e == cudaSuccess) e = adi::run_step(c);
    c.stream = own;
    if (e == cudaSuccess) e = cudaEventRecord(b->joins[i], b->streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->joins[i], 0);
  }
  return e;
}

std::string tune_key(const adi::Ctx& c) {
  std::ostringstream o;
  o << "p" << c.p << "_" << c.N[0] << "x" << c.N[1] << "x" << c.N[2] << (c.precision == ADI_PREC_FP64 ? "_f64" : "_f32");
  return o.str();
}

}  // namespace

extern "C" {

adi_status adi_set_line_tile(adi_handle h, int lines) {
  if (!h) return adi::fail_global(ADI_EINVAL, "adi_set_line_tile: NULL handle");
  if (!(lines == 0 || lines == 8 || lines == 16 || lines == 32 || lines == 64)) {
    h->err = "adi_set_line_tile: lines must be 0, 8, 16, 32 or 64";
    return ADI_EINVAL;
  }
  h->line_tile = lines;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return ADI_OK;
}

adi_status adi_batch_create(int count, const adi_instance_desc* desc, const adi_options* opt, adi_batch* out) {
  if (!out || !desc || count < 1) return adi::fail_global(ADI_EINVAL, "adi_batch_create: need count >= 1, desc, out");
  *out = nullptr;
  adi_batch b = new (std::nothrow) adi_batch_ctx();
  if (!b) return adi::fail_global(ADI_ENOMEM, "adi_batch_create: host allocation failed");
  for (int i = 0; i < count; ++i) {
    adi_handle h = nullptr;
    const adi_instance_desc& d = desc[i];
    adi_status s = adi_create(d.nx, d.ny, d.nz, d.p, d.dt, d.eps, d.mu, d.sigma, opt, &h);
    if (s != ADI_OK) {
      std::string m = std::string("adi_batch_create: instance ") + std::to_string(i) + ": " + adi_last_error(nullptr);
      free_batch(b);
      return adi::fail_global(s, m);
    }
    b->inst.push_back(h);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
  b->stream = b->own_stream;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    cudaStream_t s;
    cudaEvent_t j;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->streams.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e == cudaSuccess) b->joins.push_back(j);
  }
  if (e != cudaSuccess) {
    std::string m = std::string("adi_batch_create: ") + cudaGetErrorString(e);
    free_batch(b);
    return adi::fail_global(ADI_ECUDA, m);
  }
  *out = b;
  return ADI_OK;
}

adi_status adi_batch_set_stream(adi_batch b, void* cuda_stream) {
  if (!b) return adi::fail_global(ADI_EINVAL, "adi_batch_set_stream: NULL batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, ADI_ECUDA, std::string("adi_batch_set_stream: ") + cudaGetErrorString(e));
  b->stream = cuda_stream ? (cudaStream_t)cuda_stream : b->own_stream;
  drop_batch_graph(b);
  return ADI_OK;
}

adi_status adi_batch_handle(adi_batch b, int i, adi_handle* h) {
  if (!b || !h) return adi::fail_global(ADI_EINVAL, "adi_batch_handle: NULL argument");
  if (i < 0 || i >= (int)b->inst.size()) return bfail(b, ADI_EINVAL, "adi_batch_handle: index out of range");
  *h = b->inst[i];
  return ADI_OK;
}

adi_status adi_batch_factor(adi_batch b) {
  if (!b) return adi::fail_global(ADI_EINVAL, "adi_batch_factor: NULL batch");
  for (size_t i = 0; i < b->inst.size(); ++i) {
    adi_status s = adi_factor(b->inst[i]);
    if (s != ADI_OK) return bfail(b, s, std::string("adi_batch_factor: ") + adi_last_error(b->inst[i]));
  }
  drop_batch_graph(b);
  return ADI_OK;
}

adi_status adi_batch_step(adi_batch b, int n) {
  if (!b) return adi::fail_global(ADI_EINVAL, "adi_batch_step: NULL batch");
  if (n < 1) return bfail(b, ADI_EINVAL, "adi_batch_step: n must be >= 1");
  for (adi_handle h : b->inst)
    if (!h->factored) return bfail(b, ADI_ESTATE, "adi_batch_step: call adi_batch_factor first");
  // the instances' own work must be ordered before the batch graph
  for (adi_handle h : b->inst) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bfail(b, ADI_ECUDA, std::string("adi_batch_step: ") + cudaGetErrorString(e));
  }
  if (!b->graph) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    cudaError_t ek = e == cudaSuccess ? record_step(b) : e;
    if (e == cudaSuccess) e = cudaStreamEndCapture(b->stream, &g);
    if (ek != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bfail(b, ADI_ECUDA, std::string("adi_batch_step: capture: ") + cudaGetErrorString(ek != cudaSuccess ? ek : e));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return bfail(b, ADI_ECUDA, std::string("adi_batch_step: instantiate: ") + cudaGetErrorString(e));
    }
  }
  for (int k = 0; k < n; ++k) {
    cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) return bfail(b, ADI_ECUDA, std::string("adi_batch_step: ") + cudaGetErrorString(e));
  }
  for (adi_handle h : b->inst) h->steps_host += n;
  // later calls on an instance handle use its own stream: order them after the batch
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (adi_handle h : b->inst)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, b->fork, 0);
  if (e != cudaSuccess) return bfail(b, ADI_ECUDA, std::string("adi_batch_step: ") + cudaGetErrorString(e));
  return ADI_OK;
}

adi_status adi_batch_sync(adi_batch b) {
  if (!b) return adi::fail_global(ADI_EINVAL, "adi_batch_sync: NULL batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, ADI_ECUDA, std::string("adi_batch_sync: ") + cudaGetErrorString(e));
  for (adi_handle h : b->inst) {
    adi_status s = adi_sync(h);
    if (s != ADI_OK) return bfail(b, s, std::string("adi_batch_sync: ") + adi_last_error(h));
  }
  return ADI_OK;
}

adi_status adi_batch_autotune(adi_batch b, const char* cache_path) {
  if (!b) return adi::fail_global(ADI_EINVAL, "adi_batch_autotune: NULL batch");
  std::map<std::string, int> cache;
  if (cache_path) {
    std::ifstream f(cache_path);
    std::string key;
    int lines;
    while (f >> key >> lines) cache[key] = lines;
  }
  std::vector<std::string> fresh;
  const int cand[4] = {8, 16, 32, 64};
  for (adi_handle h : b->inst) {
    if (!h->factored) return bfail(b, ADI_ESTATE, "adi_batch_autotune: call adi_batch_factor first");
    const std::string key = tune_key(*h);
    auto it = cache.find(key);
    if (it != cache.end()) {
      adi_set_line_tile(h, it->second);
      continue;
    }
    // keep the state: trials step a copy and the original is restored
    std::vector<double> keep(6 * h->Nc);
    double t0 = 0.0;
    adi_status s = adi_fields(h, keep.data(), &t0);
    if (s != ADI_OK && s != ADI_ENUMERIC) return bfail(b, s, "adi_batch_autotune: adi_fields failed");
    float best_ms = 1e30f;
    int best = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int lines : cand) {
      adi_set_line_tile(h, lines);
      if (adi_step(h, 1) != ADI_OK) continue;  // width rejected or capture failed: skip
      cudaEventRecord(e0, h->stream);
      adi_status st = adi_step(h, 3);
      cudaEventRecord(e1, h->stream);
      if (st != ADI_OK || cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = lines;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    adi_set_line_tile(h, best);
    s = adi_set_fields(h, keep.data(), t0);  // state and time as before the trials
    if (s != ADI_OK) return bfail(b, s, "adi_batch_autotune: restoring the fields failed");
    cache[key] = best;
    fresh.push_back(key + " " + std::to_string(best));
  }
  if (cache_path && !fresh.empty()) {
    std::ofstream f(cache_path, std::ios::app);
    for (const std::string& l : fresh) f << l << "\n";
  }
  drop_batch_graph(b);
  return ADI_OK;
}

void adi_batch_destroy(adi_batch b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

}  // extern "C"
