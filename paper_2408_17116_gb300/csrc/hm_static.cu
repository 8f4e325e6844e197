// hm_farfield_static: the far-field / RCS entry point without device allocation.
//
// hm_farfield stages the observation directions and the RCS values in device
// buffers it allocates for the duration of the call.  Some callers cannot let a
// library allocate device memory while they run: a host application that has
// handed the device's memory to its own pool or allocator, or a service loop that
// forbids allocation after start-up.  This variant stages the same data in one
// file-scope device array instead, so a call allocates nothing; the caller still
// provides the solutions, the far-field output and the host RCS output.
#include <mutex>

#include "hm_internal.h"

// 65,536 doubles (512 KiB).  Every GPU that loads the library holds this array until
// the process exits.
static __device__ __align__(256) double g_farfield_scratch[HM_FARFIELD_STATIC_DOUBLES];

namespace {

const int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch[kMaxDevices] = {nullptr};

// Device address of the scratch array on device dev, which must be current.  In host code the
// array's name is a host-side stand-in, not a device address, so the address is
// looked up once per device (with that device current) and cached.
double *scratch_address(int dev)
{
    if (dev < 0 || dev >= kMaxDevices) throw HmError{HM_ERR_ARG, "device ordinal out of range for the static scratch"};
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_farfield_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw HmError{HM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)};
        }
        g_scratch[dev] = (double *)p;
    }
    return g_scratch[dev];
}

}  // namespace

extern "C" hm_status hm_farfield_static(hm_handle h, int nrhs, const void *x_dev, int nang, const double *obs_dirs,
                                        void *efar_dev, double *rcs_host)
{
    if (!h) return HM_ERR_ARG;
    try {
        if (h->state < 1) throw HmError{HM_ERR_STATE, "hm_farfield_static before hm_build_geometry"};
        if (nrhs <= 0 || nang <= 0 || !x_dev || !obs_dirs) throw HmError{HM_ERR_ARG, "bad farfield arguments"};
        const long long need = 3LL * nang + (rcs_host ? (long long)nrhs * nang : 0LL);
        if (need > HM_FARFIELD_STATIC_DOUBLES)
            throw HmError{HM_ERR_ARG, "3 nang + nrhs nang = " + std::to_string(need) +
                                          " doubles exceeds the static scratch of " +
                                          std::to_string(HM_FARFIELD_STATIC_DOUBLES)};
        // the handle's stream belongs to the device the handle was created on; the array's
        // address is looked up with that device current, before anything is copied
        int dev = 0;
        HM_CUDA(cudaGetDevice(&dev));
        if (dev != h->device)
            throw HmError{HM_ERR_STATE, "hm_farfield_static: the current device is not the handle's device"};
        double *scr = scratch_address(h->device);
        double *d_obs = scr, *d_rcs = rcs_host ? scr + 3 * (size_t)nang : nullptr;
        HM_CUDA(cudaMemcpyAsync(d_obs, obs_dirs, sizeof(double) * 3 * nang, cudaMemcpyHostToDevice, h->stream));
        if (h->dof == 4)
            launch_farfield_muller(h, nrhs, (const zc *)x_dev, nang, d_obs, (zc *)efar_dev, d_rcs);
        else
            launch_farfield(h, nrhs, (const zc *)x_dev, nang, d_obs, (zc *)efar_dev, d_rcs);
        if (rcs_host)
            HM_CUDA(cudaMemcpyAsync(rcs_host, d_rcs, sizeof(double) * (size_t)nrhs * nang, cudaMemcpyDeviceToHost,
                                    h->stream));
        HM_CUDA(cudaStreamSynchronize(h->stream));  // obs_dirs is only read during the call
        h->err.clear();
        return HM_OK;
    } catch (const HmError &e) {
        h->err = e.msg;
        return e.st;
    } catch (...) {
        h->err = "unknown error";
        return HM_ERR_CUDA;
    }
}
