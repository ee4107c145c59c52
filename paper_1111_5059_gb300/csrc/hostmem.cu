// Page-locked host buffers on transparent huge pages (dwf_host_alloc /
// dwf_host_free).
//
// A copy between the GPU and page-locked host memory translates every host
// page it touches.  On a Grace host with 64 KB base pages a 5 GB buffer is
// ~80,000 pages, and the first copy after the GPU has done other work (or
// sat idle) runs at 6-50 GB/s while the translations are fetched again; the
// same buffer backed by 512 MB transparent huge pages needs ten
// translations and copies at the link's ~190-210 GB/s from the first copy.
// So the buffer is an anonymous mapping aligned to the huge-page size,
// advised for huge pages, faulted in, then registered with the CUDA driver.
// Where the kernel offers no transparent huge pages the buffer is still
// page-locked and correct, only without the larger pages.
#include <sys/mman.h>
#include <unistd.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>

#include "dwf_internal.h"

namespace {

struct Mapping {
  void* base;
  size_t len;
};

std::mutex g_mu;
std::map<void*, Mapping> g_maps;  // user pointer -> mapping

size_t huge_page_size() {
  size_t sz = 0;
  if (FILE* f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
    unsigned long long v = 0;
    if (std::fscanf(f, "%llu", &v) == 1) sz = (size_t)v;
    std::fclose(f);
  }
  // a power of two between 64 KB and 1 GB, else 2 MB
  if (sz < (64u << 10) || sz > (1u << 30) || (sz & (sz - 1))) sz = 2u << 20;
  return sz;
}

}  // namespace

using dwf::fail;

extern "C" dwf_status dwf_host_alloc(size_t bytes, void** ptr) {
  if (!ptr) return fail(nullptr, DWF_ERR_INVALID_ARG, "dwf_host_alloc: ptr is NULL");
  *ptr = nullptr;
  if (bytes == 0) return fail(nullptr, DWF_ERR_INVALID_ARG, "dwf_host_alloc: zero bytes");
  const size_t hp = huge_page_size();
  const long ps = sysconf(_SC_PAGESIZE);
  const size_t page = ps > 0 ? (size_t)ps : 4096;
  const size_t body = (bytes + hp - 1) / hp * hp;
  if (body < bytes || body + hp < body) return fail(nullptr, DWF_ERR_INVALID_ARG, "dwf_host_alloc: size overflows");
  // over-map by one huge page so that the buffer can start on a huge-page
  // boundary; the unused head and tail go back to the system
  const size_t len = body + hp;
  void* raw = mmap(nullptr, len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (raw == MAP_FAILED) return fail(nullptr, DWF_ERR_OOM, "dwf_host_alloc: mmap failed");
  const uintptr_t r = reinterpret_cast<uintptr_t>(raw);
  const uintptr_t a = (r + hp - 1) / hp * hp;
  if (a > r) munmap(raw, a - r);
  const size_t tail = (r + len) - (a + body);
  if (tail > 0) munmap(reinterpret_cast<void*>(a + body), tail);
  void* p = reinterpret_cast<void*>(a);
#ifdef MADV_HUGEPAGE
  madvise(p, body, MADV_HUGEPAGE);  // advisory: ignored where huge pages are off
#endif
  // fault every page in (each huge page on its first touch)
  volatile unsigned char* c = static_cast<volatile unsigned char*>(p);
  for (size_t off = 0; off < body; off += page) c[off] = 0;
#ifndef MADV_COLLAPSE
#define MADV_COLLAPSE 25
#endif
  // where a fault could not get a huge page (fragmented memory), ask the
  // kernel to collapse the range synchronously; older kernels reject the
  // advice, which changes nothing
  madvise(p, body, MADV_COLLAPSE);
  const cudaError_t e = cudaHostRegister(p, body, cudaHostRegisterDefault);
  if (e != cudaSuccess) {
    munmap(p, body);
    return fail(nullptr, e == cudaErrorMemoryAllocation ? DWF_ERR_OOM : DWF_ERR_CUDA,
                std::string("dwf_host_alloc: cudaHostRegister: ") + cudaGetErrorString(e));
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_maps[p] = Mapping{p, body};
  }
  *ptr = p;
  return DWF_OK;
}

extern "C" dwf_status dwf_host_free(void* ptr) {
  if (!ptr) return DWF_OK;
  Mapping m;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_maps.find(ptr);
    if (it == g_maps.end()) return fail(nullptr, DWF_ERR_INVALID_ARG, "dwf_host_free: not a dwf_host_alloc pointer");
    m = it->second;
    g_maps.erase(it);
  }
  const cudaError_t e = cudaHostUnregister(m.base);
  munmap(m.base, m.len);
  if (e != cudaSuccess)
    return fail(nullptr, DWF_ERR_CUDA, std::string("dwf_host_free: cudaHostUnregister: ") + cudaGetErrorString(e));
  return DWF_OK;
}
