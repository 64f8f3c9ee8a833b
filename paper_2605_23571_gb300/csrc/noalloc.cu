// eda_hvp_noalloc: the batched Hessian-vector product of eda_hvp for callers
// that must not allocate device memory while they run.
//
// Who needs it: code that calls the library from inside a region where
// cudaMalloc is not allowed or not affordable -- a host thread that is
// capturing a CUDA graph in global capture mode (cudaMalloc is an illegal
// call there), an assimilation cycle that runs inside a fixed, preallocated
// memory budget shared with a forecast model, or a latency-critical loop
// that cannot afford the implicit device synchronisation an allocation may
// cause.  eda_hvp may allocate: it grows the handle's observation stash on
// the first call with more columns, and stages host arrays through temporary
// device buffers.  This variant does neither: its scratch (the per-column
// observation stash the tangent-linear sweep writes and the adjoint sweep
// reads) lives in the fixed array below, and every argument must already be
// device memory.
#include <cuda_runtime.h>

#include <atomic>

#include "handle.h"

namespace {

// Scratch of eda_hvp_noalloc: 32 MiB, shared by every call on this device
// (held by every device that loads the library, until the process exits).
constexpr long long kNoAllocScratchBytes = 32ll << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array per device, looked up once per device
// (the array's name is only a host-side stand-in in host code).  Host threads
// making their first call on one device at once may both look it up; they
// find the same address, and the atomic slot makes the publication safe.
constexpr int kMaxDevices = 64;
std::atomic<void*> g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" {

EDA_API long long eda_hvp_noalloc_capacity(int fp64) {
  return kNoAllocScratchBytes / (fp64 ? (long long)sizeof(double) : (long long)sizeof(float));
}

EDA_API int eda_hvp_noalloc(eda_handle* h, const int* member_of_col, int ncol, const double* V, double* HV,
                            int include_identity) {
  if (!h) return eda::fail(nullptr, EDA_ERR_INVALID, "handle is NULL");
  if (!h->have_traj) return eda::fail(h, EDA_ERR_STATE, "eda_hvp_noalloc before eda_set_trajectory");
  if (ncol < 0) return eda::fail(h, EDA_ERR_INVALID, "eda_hvp_noalloc: ncol < 0");
  if (ncol == 0) return EDA_OK;
  if (!member_of_col || !V || !HV)
    return eda::fail(h, EDA_ERR_INVALID, "eda_hvp_noalloc: NULL argument");
  if (!eda::is_device_ptr(member_of_col) || !eda::is_device_ptr(V) || !eda::is_device_ptr(HV))
    return eda::fail(h, EDA_ERR_INVALID, "eda_hvp_noalloc: member_of_col, V and HV must be device memory");
  const bool fp64 = (h->precision == EDA_FP64);
  const int* obs_tab = nullptr;
  const int* wtab = nullptr;
  const SweepPlan& plan = eda::hvp_plan(h, fp64, &obs_tab, &wtab);
  if (plan.ml)
    return eda::fail(h, EDA_ERR_INVALID,
                     "eda_hvp_noalloc: this state size needs multi-launch sweeps with state buffers; use eda_hvp");
  const long long need = (long long)ncol * (long long)h->p;  // stash entries
  if (need > eda_hvp_noalloc_capacity(fp64 ? 1 : 0))
    return eda::fail(h, EDA_ERR_INVALID,
                     "eda_hvp_noalloc: ncol * p = " + std::to_string(need) + " stash entries exceed the fixed " +
                         std::to_string(eda_hvp_noalloc_capacity(fp64 ? 1 : 0)) +
                         " of the 32 MiB scratch; split the columns over several calls");
  // set-up, once per device (with that device current)
  int dev = 0;
  CU(h, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return eda::fail(h, EDA_ERR_INVALID, "eda_hvp_noalloc: device index too large");
  void* scratch = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (scratch == nullptr) {
    CU(h, cudaGetSymbolAddress(&scratch, g_noalloc_scratch));
    g_scratch_ptr[dev].store(scratch, std::memory_order_release);
  }
  // The stash needs no clearing: the tangent-linear sweep writes every
  // observation entry of a column before the adjoint sweep reads it.
  if (fp64) {
    SweepArgs<double> a{};
    a.n = h->n;
    a.N = h->N;
    a.F = h->F;
    a.dt = h->dt;
    a.traj = h->traj;
    a.traj_mstride = (long long)h->trows * h->n;
    a.stages = h->stg;
    a.stage_astride = (long long)h->M * (h->N + 1) * h->n;
    a.obs_of_t = h->obs_of_t;
    a.obs_ptr = h->obs_ptr;
    a.obs_idx = h->obs_idx;
    a.rinv = h->rinv;
    a.p = h->p;
    a.w = h->w;
    a.bcoef = h->bcoef;
    a.nos = h->nos;
    a.obs_tab = obs_tab;
    a.wtab = wtab;
    a.mode = eda::MODE_HVP;
    a.ncol = ncol;
    a.col_member = member_of_col;
    a.M = h->M;
    a.V = V;
    a.v_stride = h->n;
    a.OUT = HV;
    a.out_stride = h->n;
    a.stash = static_cast<double*>(scratch);
    a.stash_stride = h->p;
    a.include_identity = include_identity ? 1 : 0;
    CU(h, eda::launch_sweep<double>(a, plan, h->st));
  } else {
    SweepArgs<float> a{};
    a.n = h->n;
    a.N = h->N;
    a.F = (float)h->F;
    a.dt = (float)h->dt;
    a.traj = h->traj32;
    a.traj_mstride = (long long)h->trows * h->n;
    a.obs_of_t = h->obs_of_t;
    a.obs_ptr = h->obs_ptr;
    a.obs_idx = h->obs_idx;
    a.rinv = h->rinv32;
    a.p = h->p;
    a.w = h->w;
    a.bcoef = h->bcoef32;
    a.nos = h->nos;
    a.obs_tab = obs_tab;
    a.wtab = wtab;
    a.mode = eda::MODE_HVP;
    a.ncol = ncol;
    a.col_member = member_of_col;
    a.M = h->M;
    a.V64 = V;
    a.v_stride = h->n;
    a.OUT64 = HV;
    a.out_stride = h->n;
    a.stash = static_cast<float*>(scratch);
    a.stash_stride = h->p;
    a.include_identity = include_identity ? 1 : 0;
    CU(h, eda::launch_sweep<float>(a, plan, h->st));
  }
  return EDA_OK;
}

}  // extern "C"
