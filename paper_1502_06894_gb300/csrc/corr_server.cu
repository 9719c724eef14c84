// corr_server.cu -- the continuous-batching correlation server behind the
// corr_server_* entry points of include/corr.h.
//
// One worker thread owns the device work.  Submitted jobs (a scan whose
// samples are already in device memory, a precision, a rotation form and a
// number of integrations) wait in a FIFO queue; the worker admits them while
// the device memory they need (corr_device_bytes plus their output buffers)
// stays within the cap minus the reserve, so a job that arrives while others
// are on the GPU joins as soon as memory frees up.  Every step advances every
// admitted job by one integration in one CUDA graph (corr_batch_run), copies
// each job's visibilities to its pinned host buffer, and hands them to the
// job's callback on the worker thread.  A job's latency runs from its
// submission to the end of its last callback.
//
// The correlation itself is the FX path of the paper (Abstract: Fourier
// transform, then cross-multiply) as the handle API computes it; the paper
// has no serving layer.
#include "../../include/corr.h"
#include "corr_internal.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t id = 0;
  // copies of the caller's descriptor
  int S = 0, nsub = 0, npol = 0, nchan = 0;
  double fs = 0.0, tint = 0.0;
  float lut[4] = {};
  std::vector<double> nu0;
  std::vector<int> nseg;
  std::vector<double> t0, coeffs;  // [S][64], [S][64][6]
  std::vector<const void*> bytes;
  std::vector<size_t> nbytes;
  std::vector<int64_t> first;
  int precision = CORR_PREC_FP32, rotation = CORR_ROT_POST_F;
  int64_t nint = 0;
  corr_result_fn fn = nullptr;
  void* user = nullptr;
  Clock::time_point submitted;
  // once the worker has looked at it
  corr_t* h = nullptr;
  size_t need = 0;  // device bytes while admitted (handle work buffers + outputs)
  size_t bytes_held = 0;
  float* dev_out = nullptr;
  double* dev_w = nullptr;
  float* host_out = nullptr;
  double* host_w = nullptr;
  int64_t done = 0;
  double samples_per_integration = 0.0;
};

}  // namespace

struct corr_server_s {
  int dev = 0;
  size_t cap = 0, reserve = 0;
  std::mutex mu;
  std::condition_variable cv, cv_idle;
  std::deque<Job*> queue;     // submitted, not yet admitted
  std::vector<Job*> active;   // owned by the worker
  bool stop = false;
  int64_t next_id = 1;
  int64_t submitted = 0, finished = 0;
  std::vector<double> latencies;  // seconds, of finished jobs
  double samples = 0.0;           // station-samples of finished integrations
  Clock::time_point first_submit, last_finish;
  bool any_submit = false;
  size_t in_use = 0;
  cudaStream_t stream = nullptr;
  std::thread worker;
};

namespace {

bool desc_ok(const corr_job* j) {
  const corr_scan_desc& d = j->scan;
  if (d.stations < 1 || d.stations > corr::kMaxStations || d.pols < 1 || d.pols > 2 || d.subbands < 1 ||
      d.subbands * d.pols > 32 || d.nchan < 4 || d.nchan > 8192 || (d.nchan & (d.nchan - 1)) || !(d.fs_hz > 0) ||
      !(d.tint_s > 0))
    return false;
  if (!d.nu0_hz || !d.nseg || !d.seg_t0 || !d.seg_coeffs || !d.dev_bytes || !d.nbytes || !d.first_sample) return false;
  for (int s = 0; s < d.stations; ++s) {
    if (d.nseg[s] < 1 || d.nseg[s] > corr::kMaxSegs) return false;
    if (!d.dev_bytes[s] || ((uintptr_t)d.dev_bytes[s] & 15) || (d.nbytes[s] & 3)) return false;
  }
  if (j->precision < CORR_PREC_FP32 || j->precision > CORR_PREC_FP8_TC) return false;
  if (j->rotation != CORR_ROT_POST_F && j->rotation != CORR_ROT_PRE_F) return false;
  if (j->integrations < 1) return false;
  return true;
}

// A handle for the job, configured and with its samples attached; its device
// bytes (before any device allocation) in *bytes.
int make_handle(Job* j, size_t* bytes) {
  corr_t* h = nullptr;
  int rc = corr_create(&h, j->S, j->nsub, j->npol, j->nchan, j->tint);
  if (rc) return rc;
  if ((rc = corr_set_format(h, j->fs, j->lut)) || (rc = corr_set_precision(h, j->precision)) ||
      (rc = corr_set_fringe_rotation(h, j->rotation))) {
    corr_destroy(h);
    return rc;
  }
  for (int sb = 0; sb < j->nsub && !rc; ++sb) rc = corr_set_sky_freq(h, sb, j->nu0[sb]);
  for (int s = 0; s < j->S && !rc; ++s) {
    for (int q = 0; q < j->nseg[s] && !rc; ++q)
      rc = corr_set_delay_poly(h, s, j->t0[(size_t)s * corr::kMaxSegs + q],
                               &j->coeffs[((size_t)s * corr::kMaxSegs + q) * 6]);
    if (!rc) rc = corr_set_stream_start(h, s, j->first[s]);
    if (!rc) rc = corr_attach_samples_device(h, s, j->bytes[s], j->nbytes[s]);
  }
  if (!rc) rc = corr_flush(h);
  if (!rc) rc = corr_device_bytes(h, bytes);
  if (rc) {
    corr_destroy(h);
    return rc;
  }
  j->h = h;
  return CORR_OK;
}

void release(corr_server_s* sv, Job* j) {
  if (j->h) corr_destroy(j->h);
  cudaFree(j->dev_out);
  cudaFree(j->dev_w);
  cudaFreeHost(j->host_out);
  cudaFreeHost(j->host_w);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->in_use -= j->bytes_held;
  }
  delete j;
}

void fail_job(corr_server_s* sv, Job* j, int status) {
  if (j->fn) j->fn(j->user, j->id, j->done, nullptr, nullptr, status);
  release(sv, j);
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->finished += 1;
  sv->cv_idle.notify_all();
}

// Admit queued jobs (first come, first served) while they fit.
void admit(corr_server_s* sv) {
  const size_t budget = sv->cap - sv->reserve;
  for (;;) {
    Job* j = nullptr;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (sv->queue.empty()) return;
      j = sv->queue.front();
    }
    int rc = CORR_OK;
    const size_t nbl = (size_t)j->S * (j->S + 1) / 2;
    const size_t out_bytes = nbl * j->nsub * j->npol * j->nchan * 2 * sizeof(float);
    if (!j->h) {  // first look: the handle and its memory estimate (kept while the job waits)
      rc = make_handle(j, &j->need);
      j->need += out_bytes + nbl * sizeof(double);
    }
    const size_t need = j->need;
    const bool fits_ever = need <= budget;
    bool fits_now;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      fits_now = sv->in_use + need <= budget;
      if (rc == CORR_OK && fits_ever && fits_now) {
        sv->queue.pop_front();
        sv->in_use += need;
        j->bytes_held = need;
      } else if (rc != CORR_OK || !fits_ever) {
        sv->queue.pop_front();
      }
    }
    if (rc != CORR_OK || !fits_ever) {
      fail_job(sv, j, rc != CORR_OK ? rc : CORR_ENOMEM);
      continue;
    }
    if (!fits_now) return;  // wait for memory: the job stays at the head of the queue
    cudaError_t e = cudaMalloc((void**)&j->dev_out, out_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&j->dev_w, nbl * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&j->host_out, out_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&j->host_w, nbl * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(j->dev_w, 0, nbl * sizeof(double), sv->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail_job(sv, j, CORR_ENOMEM);
      continue;
    }
    j->samples_per_integration = (double)j->S * j->nsub * j->npol * (double)llround(j->fs * j->tint);
    sv->active.push_back(j);
  }
}

// One step: the next integration of every admitted job in one graph, results
// to the host, callbacks, retirement of finished jobs.
void step(corr_server_s* sv) {
  const int n = (int)sv->active.size();
  std::vector<corr_t*> hs(n);
  std::vector<float*> outs(n);
  std::vector<double*> ws(n);
  for (int q = 0; q < n; ++q) {
    hs[q] = sv->active[q]->h;
    outs[q] = sv->active[q]->dev_out;
    ws[q] = sv->active[q]->dev_w;
  }
  int rc = corr_batch_run(hs.data(), n, outs.data(), ws.data(), sv->stream);
  cudaError_t e = cudaSuccess;
  if (rc == CORR_OK) {
    for (int q = 0; q < n && e == cudaSuccess; ++q) {
      Job* j = sv->active[q];
      const size_t nbl = (size_t)j->S * (j->S + 1) / 2;
      e = cudaMemcpyAsync(j->host_out, j->dev_out, nbl * j->nsub * j->npol * j->nchan * 2 * sizeof(float),
                          cudaMemcpyDeviceToHost, sv->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(j->host_w, j->dev_w, nbl * sizeof(double), cudaMemcpyDeviceToHost, sv->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->stream);
    if (e != cudaSuccess) rc = CORR_ECUDA;
  }
  std::vector<Job*> keep;
  for (int q = 0; q < n; ++q) {
    Job* j = sv->active[q];
    if (rc != CORR_OK) {
      fail_job(sv, j, rc);
      continue;
    }
    if (j->fn) j->fn(j->user, j->id, j->done, j->host_out, j->host_w, CORR_OK);
    j->done += 1;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->samples += j->samples_per_integration;
    }
    if (j->done < j->nint) {
      keep.push_back(j);
      continue;
    }
    const double lat = std::chrono::duration<double>(Clock::now() - j->submitted).count();
    release(sv, j);
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->latencies.push_back(lat);
    sv->finished += 1;
    sv->last_finish = Clock::now();
    sv->cv_idle.notify_all();
  }
  sv->active.swap(keep);
}

void worker_main(corr_server_s* sv) {
  cudaSetDevice(sv->dev);
  if (cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    sv->stream = nullptr;
  }
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait(lk, [&] { return sv->stop || !sv->queue.empty() || !sv->active.empty(); });
      if (sv->stop && sv->queue.empty() && sv->active.empty()) break;
    }
    admit(sv);
    if (sv->active.empty()) {
      // nothing fits yet and nothing runs: wait for a submission or a stop
      std::unique_lock<std::mutex> lk(sv->mu);
      if (!sv->stop) sv->cv.wait_for(lk, std::chrono::milliseconds(50));
      if (sv->stop) break;
      continue;
    }
    step(sv);
  }
  // stopping: fail what is left
  for (Job* j : sv->active) fail_job(sv, j, CORR_ESTATE);
  sv->active.clear();
  for (;;) {
    Job* j = nullptr;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (sv->queue.empty()) break;
      j = sv->queue.front();
      sv->queue.pop_front();
    }
    fail_job(sv, j, CORR_ESTATE);
  }
  if (sv->stream) cudaStreamDestroy(sv->stream);
}

}  // namespace

extern "C" {

int corr_server_start(corr_server_t** out, size_t hbm_cap_bytes, size_t reserve_bytes) {
  if (!out) return CORR_EINVAL;
  *out = nullptr;
  if (hbm_cap_bytes == 0 || reserve_bytes >= hbm_cap_bytes) return CORR_EINVAL;
  corr_server_s* sv = new (std::nothrow) corr_server_s();
  if (!sv) return CORR_ENOMEM;
  if (cudaGetDevice(&sv->dev) != cudaSuccess) {
    cudaGetLastError();
    sv->dev = 0;
  }
  sv->cap = hbm_cap_bytes;
  sv->reserve = reserve_bytes;
  try {
    sv->worker = std::thread(worker_main, sv);
  } catch (...) {
    delete sv;
    return CORR_ENOMEM;
  }
  *out = sv;
  return CORR_OK;
}

int corr_server_submit(corr_server_t* sv, const corr_job* job, corr_result_fn fn, void* user, int64_t* job_id) {
  if (!sv || !job || !desc_ok(job)) return CORR_EINVAL;
  const corr_scan_desc& d = job->scan;
  Job* j = new (std::nothrow) Job();
  if (!j) return CORR_ENOMEM;
  j->S = d.stations;
  j->nsub = d.subbands;
  j->npol = d.pols;
  j->nchan = d.nchan;
  j->fs = d.fs_hz;
  j->tint = d.tint_s;
  for (int q = 0; q < 4; ++q) j->lut[q] = d.lut[q];
  j->nu0.assign(d.nu0_hz, d.nu0_hz + d.subbands);
  j->nseg.assign(d.nseg, d.nseg + d.stations);
  j->t0.assign(d.seg_t0, d.seg_t0 + (size_t)d.stations * corr::kMaxSegs);
  j->coeffs.assign(d.seg_coeffs, d.seg_coeffs + (size_t)d.stations * corr::kMaxSegs * 6);
  j->bytes.assign(d.dev_bytes, d.dev_bytes + d.stations);
  j->nbytes.assign(d.nbytes, d.nbytes + d.stations);
  j->first.assign(d.first_sample, d.first_sample + d.stations);
  j->precision = job->precision;
  j->rotation = job->rotation;
  j->nint = job->integrations;
  j->fn = fn;
  j->user = user;
  j->submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
      delete j;
      return CORR_ESTATE;
    }
    j->id = sv->next_id++;
    if (!sv->any_submit) {
      sv->any_submit = true;
      sv->first_submit = j->submitted;
    }
    sv->submitted += 1;
    sv->queue.push_back(j);
    if (job_id) *job_id = j->id;
  }
  sv->cv.notify_all();
  return CORR_OK;
}

int corr_server_stats(corr_server_t* sv, double* p50_s, double* p99_s, double* samples_per_s, int64_t* jobs_done) {
  if (!sv) return CORR_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  std::vector<double> lat = sv->latencies;
  std::sort(lat.begin(), lat.end());
  // nearest rank
  auto pct = [&](double p) -> double {
    if (lat.empty()) return 0.0;
    size_t k = (size_t)std::ceil(p * (double)lat.size());
    if (k < 1) k = 1;
    return lat[std::min(k, lat.size()) - 1];
  };
  if (p50_s) *p50_s = pct(0.50);
  if (p99_s) *p99_s = pct(0.99);
  if (samples_per_s) {
    const double span = sv->any_submit && sv->finished > 0
                            ? std::chrono::duration<double>(sv->last_finish - sv->first_submit).count()
                            : 0.0;
    *samples_per_s = span > 0 ? sv->samples / span : 0.0;
  }
  if (jobs_done) *jobs_done = sv->finished;
  return CORR_OK;
}

int corr_server_wait(corr_server_t* sv, double timeout_s) {
  if (!sv) return CORR_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto idle = [&] { return sv->finished == sv->submitted; };
  if (timeout_s < 0) {
    sv->cv_idle.wait(lk, idle);
    return CORR_OK;
  }
  return sv->cv_idle.wait_for(lk, std::chrono::duration<double>(timeout_s), idle) ? CORR_OK : CORR_ETIMEOUT;
}

void corr_server_stop(corr_server_t* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  delete sv;
}

}  // extern "C"
