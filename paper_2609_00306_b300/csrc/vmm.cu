// vmm.cu -- device arrays that grow in place (CUDA virtual memory management).
//
// The vector store of a decomposition grows with the vector count M, which is
// known only at the end.  A cudaMalloc'd array can only grow by allocating a
// larger one and copying, which needs the old and the new array at once (at
// N = 2000 that would be about twice the 140 GB the decomposition holds).
// Here a virtual address range large enough for the largest allowed M is
// reserved once, and physical memory is mapped into it, in granules, only as
// the vectors are produced: the array never moves, growing it copies nothing,
// and the memory held is what has been mapped.
#include <cuda.h>
#include <mutex>
#include <string>
#include "internal.cuh"

namespace cd {

namespace {
// The driver entry points are looked up through the runtime (no link-time
// dependency on the driver library, so the library also loads where no GPU
// driver is installed).
struct DriverVmm {
  decltype(&cuMemGetAllocationGranularity) granularity = nullptr;
  decltype(&cuMemAddressReserve) reserve = nullptr;
  decltype(&cuMemAddressFree) address_free = nullptr;
  decltype(&cuMemCreate) create = nullptr;
  decltype(&cuMemRelease) release = nullptr;
  decltype(&cuMemMap) map = nullptr;
  decltype(&cuMemUnmap) unmap = nullptr;
  decltype(&cuMemSetAccess) set_access = nullptr;
  bool ok = false;
};
template <class F>
bool lookup(const char* name, F* fn) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return false;
  }
  *fn = (F)p;
  return true;
}
const DriverVmm& drv() {
  static DriverVmm d;
  static std::once_flag once;
  std::call_once(once, [] {
    d.ok = lookup("cuMemGetAllocationGranularity", &d.granularity) && lookup("cuMemAddressReserve", &d.reserve) &&
           lookup("cuMemAddressFree", &d.address_free) && lookup("cuMemCreate", &d.create) &&
           lookup("cuMemRelease", &d.release) && lookup("cuMemMap", &d.map) && lookup("cuMemUnmap", &d.unmap) &&
           lookup("cuMemSetAccess", &d.set_access);
  });
  return d;
}
int cu_fail(CUresult r, const char* what) {
  set_error(std::string(what) + " failed (CUresult " + std::to_string((int)r) + ")");
  return r == CUDA_ERROR_OUT_OF_MEMORY ? CD_ENOMEM : CD_ECUDA;
}
}  // namespace

int VmArray::reserve(size_t bytes) {
  release();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); set_error("cudaGetDevice failed"); return CD_ECUDA; }
  cudaFree(nullptr);  // the primary context exists before the driver calls below
  const DriverVmm& D = drv();
  if (!D.ok) { set_error("CUDA virtual memory entry points unavailable"); return CD_ECUDA; }
  device = dev;
  CUmemAllocationProp prop = {};
  prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
  prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  prop.location.id = dev;
  CUresult r = D.granularity(&gran, &prop, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED);
  if (r != CUDA_SUCCESS) return cu_fail(r, "cuMemGetAllocationGranularity");
  reserved = (bytes + gran - 1) / gran * gran;
  if (reserved == 0) reserved = gran;
  CUdeviceptr p = 0;
  r = D.reserve(&p, reserved, 0, 0, 0);
  if (r != CUDA_SUCCESS) { reserved = 0; return cu_fail(r, "cuMemAddressReserve"); }
  base = (void*)p;
  mapped = 0;
  return CD_OK;
}

int VmArray::grow(size_t bytes) {
  if (bytes <= mapped) return CD_OK;
  if (!base) { set_error("VmArray: not reserved"); return CD_EINVAL; }
  const size_t want = (bytes + gran - 1) / gran * gran;
  if (want > reserved) { set_error("VmArray: growth beyond the reserved range"); return CD_ENOMEM; }
  const size_t add = want - mapped;
  const DriverVmm& D = drv();
  CUmemAllocationProp prop = {};
  prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
  prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  prop.location.id = device;
  CUmemGenericAllocationHandle h = 0;
  CUresult r = D.create(&h, add, &prop, 0);
  if (r != CUDA_SUCCESS) return cu_fail(r, "cuMemCreate");
  const CUdeviceptr at = (CUdeviceptr)base + mapped;
  r = D.map(at, add, 0, h, 0);
  if (r != CUDA_SUCCESS) { D.release(h); return cu_fail(r, "cuMemMap"); }
  CUmemAccessDesc ad = {};
  ad.location = prop.location;
  ad.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
  r = D.set_access(at, add, &ad, 1);
  if (r != CUDA_SUCCESS) { D.unmap(at, add); D.release(h); return cu_fail(r, "cuMemSetAccess"); }
  pieces.push_back({mapped, add, (unsigned long long)h});
  mapped = want;
  return CD_OK;
}

void VmArray::release() {
  if (!base) return;
  // work queued on the array must be done before it is unmapped
  cudaDeviceSynchronize();
  const DriverVmm& D = drv();
  for (auto it = pieces.rbegin(); it != pieces.rend(); ++it) {
    D.unmap((CUdeviceptr)base + it->offset, it->size);
    D.release((CUmemGenericAllocationHandle)it->handle);
  }
  pieces.clear();
  D.address_free((CUdeviceptr)base, reserved);
  base = nullptr;
  reserved = mapped = 0;
}

}  // namespace cd
