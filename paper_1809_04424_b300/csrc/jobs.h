// jobs.h -- the batch engine as asynchronous jobs, for the request server.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/vr.h"

namespace vr {

struct JobCloud {
  int64_t pt;      // first row in the job's point buffer
  int32_t n, maxdim;
  double maxrad;
};

struct Job;  // one batch: size -> build -> finish, each step ending on an event

// Validate and describe the clouds; on error returns NULL with *err set.
// `pinned` (optional, job_pinned_bytes(n) bytes of page-locked host memory
// that outlives the job) makes every host<->device copy of the job
// asynchronous; without it the copies of per-cloud sizes block.
Job *job_create(cudaStream_t s, const void *dpts, int d, vr_dtype dtype, const std::vector<JobCloud> &clouds,
                void *pinned, vr_status *err);
size_t job_pinned_bytes(size_t n_clouds);
vr_status job_size_async(Job *j);
// Admits clouds while their exact output bytes fit `budget` (the first
// always); the indices of the others are appended to `deferred`.
vr_status job_build_async(Job *j, int64_t budget, std::vector<int> *deferred);
bool job_ready(Job *j);                        // has the last step's event completed?
int64_t job_out_bytes(Job *j);                 // admitted output bytes
// `detach`: results (and their shared arenas) use the legacy stream from now
// on, so they outlive the job's stream.
void job_finish(Job *j, std::vector<vr_complex *> &results, std::vector<vr_status> &status, bool detach);
void job_destroy(Job *j);
bool fused_fits(int n, int d);                 // can the batch kernels take this cloud?
void inject_admission_refusals(int64_t k);     // test hook: refuse the next k admissions outright
vr_status check_cloud_args(int64_t n, int d, vr_dtype dtype, int maxdim, double maxrad);

}  // namespace vr
