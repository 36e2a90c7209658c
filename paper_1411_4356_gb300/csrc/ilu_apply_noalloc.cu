// om_ilu_apply_noalloc: the preconditioner solve z = (L U)^{-1} v (or its
// conjugate transpose) without any device allocation.
//
// om_ilu_apply obtains its complex64 work vector from cudaMallocAsync on
// every call.  Some callers cannot do that: code whose device memory is owned
// by another allocator (a framework's caching pool that must see every byte),
// and code on a latency-critical path that must not enter the allocator or
// risk the implicit device synchronisation of cudaMalloc/cudaFree.  This
// variant takes its scratch -- a complex64 work vector of up to kMaxRows
// entries -- from a file-scope __device__ array instead.
//
// That array exists once per device that loads the library and lives until
// the process exits (8 MiB).  Every call shares it and it keeps the previous
// call's contents; nothing in it has to start at zero (each call writes the
// whole work vector before reading it), and two calls whose work overlaps on
// the GPU race on the same scratch (for example two host threads calling it
// on two streams).  In host code the array's name is only a host-side
// stand-in, so the first call on each device looks up its device address
// with cudaGetSymbolAddress (with that device current) and caches it.  Every
// call ends by synchronising its stream, so a call returns with its result
// written.
#include <mutex>
#include <vector>

#include "common.cuh"

namespace omss {
namespace {

constexpr int64_t kMaxRows = int64_t(1) << 20;  // 1,048,576 rows
constexpr size_t kWorkBytes = sizeof(float2) * kMaxRows;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kWorkBytes];

struct DeviceScratch {
    float2 *work = nullptr;
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
        OM_REQUIRE(!fp64 || M->has_fp64, "om_ilu_apply_noalloc: factor built without complex128 sweep data");
        cudaStream_t s = as_stream(stream);
        const DeviceScratch d = scratch_for_current_device();
        precond_apply(*M, conj_transpose, fp64, reinterpret_cast<const double2 *>(v), reinterpret_cast<double2 *>(z),
                      d.work, s, /*allow_split=*/false);
        OM_CUDA_TRY(cudaStreamSynchronize(s));
    });
}
