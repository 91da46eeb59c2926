// Page-locked host buffers for moving operands and results across the
// host link (magnus_host_alloc / magnus_host_free).
//
// The copies of a product's inputs and of C run at the host link's speed
// only when the page-locked memory maps to few, large pages: pinned memory
// handed out in small pages after other processes have fragmented host
// memory copies several times slower (the device's address translation of
// host memory then misses constantly).  These buffers are anonymous mappings
// advised to use transparent huge pages (the kernel compacts memory to grant
// them when its defrag policy honours the advice), touched once so every page
// exists, then registered with the CUDA driver as page-locked.  A huge page
// can only back a range aligned to its size, so the mapping is placed on a
// huge-page boundary and rounded up to whole huge pages (up to one huge page
// of extra memory per buffer).
#include <errno.h>
#include <stdio.h>
#include <string.h>
#include <sys/mman.h>
#include <unistd.h>

#include <thread>
#include <vector>

#include "internal.h"

extern "C" {

// Size of a transparent huge page (bytes), 0 if unknown.
static size_t thp_size() {
  static size_t v = [] {
    size_t r = 0;
    FILE* f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r");
    if (f) {
      unsigned long long x = 0;
      if (fscanf(f, "%llu", &x) == 1) r = (size_t)x;
      fclose(f);
    }
    return r;
  }();
  return v;
}

// Length of the mapping that backs a buffer of `bytes`.
static size_t mapped_len(size_t bytes) {
  const size_t hp = thp_size();
  return hp ? (bytes + hp - 1) / hp * hp : bytes;
}

int magnus_host_alloc(size_t bytes, void** ptr) {
  if (!ptr || bytes == 0) return MAGNUS_INVALID_ARG;
  *ptr = nullptr;
  const size_t hp = thp_size();
  const size_t len = mapped_len(bytes);
  // map one huge page more, then trim the unaligned head and the tail
  const size_t span = len + hp;
  void* raw = mmap(nullptr, span, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (raw == MAP_FAILED) return MAGNUS_OUT_OF_MEMORY;
  uintptr_t a = (uintptr_t)raw;
  uintptr_t start = hp ? (a + hp - 1) / hp * hp : a;
  if (start > a) munmap(raw, start - a);
  if (a + span > start + len) munmap((void*)(start + len), a + span - (start + len));
  void* p = (void*)start;
#ifdef MADV_HUGEPAGE
  madvise(p, len, MADV_HUGEPAGE);  // advice only: small pages still work
#endif
  // first touch, one write per 4 KB, split over a few threads
  const long page = sysconf(_SC_PAGESIZE) > 0 ? sysconf(_SC_PAGESIZE) : 4096;
  unsigned nt = std::thread::hardware_concurrency();
  nt = nt < 1 ? 1 : (nt > 8 ? 8 : nt);
  const size_t per = ((bytes / nt) / (size_t)page + 1) * (size_t)page;
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) {
    const size_t lo = t * per;
    if (lo >= bytes) break;
    const size_t hi = lo + per < bytes ? lo + per : bytes;
    th.emplace_back([p, lo, hi, page]() {
      volatile unsigned char* b = static_cast<unsigned char*>(p);
      for (size_t o = lo; o < hi; o += (size_t)page) b[o] = 0;
    });
  }
  for (auto& t : th) t.join();
  const cudaError_t e = cudaHostRegister(p, bytes, cudaHostRegisterDefault);
  if (e != cudaSuccess) {
    munmap(p, len);
    return magnus::api_cuda_fail(e, "cudaHostRegister");
  }
  *ptr = p;
  return MAGNUS_OK;
}

int magnus_host_free(void* ptr, size_t bytes) {
  if (!ptr) return MAGNUS_OK;
  const cudaError_t e = cudaHostUnregister(ptr);
  munmap(ptr, mapped_len(bytes));
  return e == cudaSuccess ? MAGNUS_OK : magnus::api_cuda_fail(e, "cudaHostUnregister");
}

}  // extern "C"
