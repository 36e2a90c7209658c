// om_ilu_apply_noalloc: the preconditioner solve z = (L U)^{-1} v (or its
// conjugate transpose) without any device allocation.
//
// om_ilu_apply obtains its complex64 work vector from cudaMallocAsync on
// every call.  Some callers cannot do that: code whose device memory is owned
// by another allocator (a framework's caching pool that must see every byte),
// and code on a latency-critical path that must not enter the allocator or
// risk the implicit device synchronisation of cudaMalloc/cudaFree.  This
// variant takes its scratch -- a complex64 work vector of up to kMaxRows
// entries and one status word -- from a file-scope __device__ array instead.
//
// That array exists once per device that loads the library and lives until
// the process exits (8 MiB + 256 bytes).  Every call shares it and it keeps
// the previous call's contents, so the status word is cleared on each call
// (the work vector is fully overwritten before it is read), and two calls
// whose work overlaps on the GPU race on the same scratch.  In host code the
// array's name is only a host-side stand-in, so the first call on each device
// looks up its device address with cudaGetSymbolAddress (with that device
// current) and caches it; make that first call before any stream capture.
#include <mutex>
#include <vector>

#include "common.cuh"

namespace omss {
namespace {

constexpr int64_t kMaxRows = int64_t(1) << 20;  // 1,048,576 rows
constexpr size_t kWorkBytes = sizeof(float2) * kMaxRows;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kWorkBytes + 256];

struct DeviceScratch {
    float2 *work = nullptr;
    int *status = nullptr;
};

std::mutex g_scratch_mu;
std::vector<DeviceScratch> g_scratch_by_device;

DeviceScratch scratch_for_current_device() {
    int dev = 0;
    OM_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if ((int)g_scratch_by_device.size() <= dev) g_scratch_by_device.resize(dev + 1);
    DeviceScratch &d = g_scratch_by_device[dev];
    if (!d.work) {
        void *base = nullptr;
        OM_CUDA_TRY(cudaGetSymbolAddress(&base, g_noalloc_scratch));
        d.work = reinterpret_cast<float2 *>(base);
        d.status = reinterpret_cast<int *>(static_cast<unsigned char *>(base) + kWorkBytes);
    }
    return d;
}

}  // namespace
}  // namespace omss

using namespace omss;

extern "C" om_status om_ilu_apply_noalloc(const om_ilu *M, int32_t flags, const double *v, double *z,
                                          void *stream) {
    return guarded([&] {
        OM_REQUIRE(M && v && z, "om_ilu_apply_noalloc: NULL argument");
        OM_REQUIRE(M->N <= kMaxRows, "om_ilu_apply_noalloc: the factor has more rows than the static scratch "
                                     "holds (1048576); use om_ilu_apply");
        const bool conj_transpose = (flags & 2) != 0;
        const bool fp64 = (flags & 1) != 0;
        OM_REQUIRE(!conj_transpose || M->has_transpose,
                   "om_ilu_apply_noalloc: factor built without conjugate transposes");
        cudaStream_t s = as_stream(stream);
        const DeviceScratch d = scratch_for_current_device();
        const double2 *vv = reinterpret_cast<const double2 *>(v);
        double2 *zz = reinterpret_cast<double2 *>(z);
        OM_CUDA_TRY(cudaMemsetAsync(d.status, 0, sizeof(int), s));
        if (fp64) {
            if (!conj_transpose) {
                sweep_c128(M->L, true, nullptr, vv, zz, d.status, 0, s);
                sweep_c128(M->U, false, M->dinv.p, zz, zz, d.status, 0, s);
            } else {
                sweep_c128(M->UH, true, M->dinvh.p, vv, zz, d.status, 0, s);
                sweep_c128(M->LH, false, nullptr, zz, zz, d.status, 0, s);
            }
        } else {
            to_c64(vv, M->N, d.work, s);
            if (!conj_transpose) {
                sweep_c64(M->L, true, nullptr, d.work, d.work, d.status, 0, s);
                sweep_c64(M->U, false, M->dinv32.p, d.work, d.work, d.status, 0, s);
            } else {
                sweep_c64(M->UH, true, M->dinvh32.p, d.work, d.work, d.status, 0, s);
                sweep_c64(M->LH, false, nullptr, d.work, d.work, d.status, 0, s);
            }
            to_c128(d.work, M->N, zz, s);
        }
        int flag = 0;
        OM_CUDA_TRY(cudaMemcpyAsync(&flag, d.status, sizeof(int), cudaMemcpyDeviceToHost, s));
        OM_CUDA_TRY(cudaStreamSynchronize(s));
        if (flag) throw Error{OM_ETIMEOUT, "triangular sweep wait timed out"};
    });
}
