// ipg_host_alloc / ipg_host_free: page-locked host buffers for the host-array entry points.
//
// ipg_graph_create and the other host-buffer calls copy with cudaMemcpyAsync, whose
// speed depends on how the host array is backed.  Measured on GB300 machines: uploading a
// 15 GB graph from the CUDA runtime's own page-locked memory took 150 ms in a fresh
// machine but 260-340 ms once other processes had churned the machine's memory (a GPU
// test suite run before), while the same upload from the buffers made here stayed at
// 150-160 ms in both states.  The likely cause is that the runtime's buffers then land
// on scattered base pages and the copy engines pay an address translation per page.
//
// These buffers are anonymous mappings aligned to the transparent huge page size and
// advised MADV_HUGEPAGE before their first touch, so the kernel backs them with huge
// pages where it can (compacting memory if it must).  Where the page faults still got
// base pages (memory fragmented by earlier processes), MADV_COLLAPSE asks the kernel
// to gather them into huge pages synchronously; kernels without it ignore the request.
// The buffers are then registered with cudaHostRegister (portable to every context).
// On one box, after the GPU test suite, an upload from base-page buffers ran at
// 14.5 GB/s against 170-210 GB/s from huge pages.  Small requests (below one huge page)
// are page aligned only.  Where the kernel has no transparent huge pages the advice is
// ignored and the buffer is an ordinary page-locked mapping.
#include <sys/mman.h>
#include <unistd.h>

#ifndef MADV_COLLAPSE
#define MADV_COLLAPSE 25  // Linux 6.1: collapse the range into transparent huge pages now
#endif

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <unordered_map>

#include "ipg_internal.cuh"

namespace ipg {
namespace {

struct HostBlock {
    void* map;   // start of the mapping that remains after trimming (== the user pointer)
    size_t len;  // its length
};

std::mutex g_host_mu;
std::unordered_map<void*, HostBlock>& host_blocks() {
    static auto* m = new std::unordered_map<void*, HostBlock>();  // never destroyed: frees may come at exit
    return *m;
}

size_t base_page() {
    long p = sysconf(_SC_PAGESIZE);
    return p > 0 ? (size_t)p : 4096;
}

size_t huge_page() {
    static const size_t v = [] {
        size_t s = (size_t)2 << 20;
        if (FILE* f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
            unsigned long long x = 0;
            if (std::fscanf(f, "%llu", &x) == 1 && x >= 4096 && x <= (1ull << 30) && (x & (x - 1)) == 0)
                s = (size_t)x;
            std::fclose(f);
        }
        return s;
    }();
    return v;
}

}  // namespace
}  // namespace ipg

using namespace ipg;

extern "C" ipg_status ipg_host_alloc(size_t bytes, void** out) {
    if (!out) return set_error(IPG_EINVAL, "ipg_host_alloc: out is NULL");
    *out = nullptr;
    if (bytes == 0) return IPG_OK;
    const size_t page = base_page();
    const size_t granule = bytes >= huge_page() ? huge_page() : page;
    if (bytes > SIZE_MAX / 2 - 2 * granule)
        return set_error(IPG_ENOMEM, "ipg_host_alloc: %zu bytes is too large", bytes);
    const size_t len = (bytes + granule - 1) / granule * granule;
    const size_t map_len = len + (granule > page ? granule : 0);  // slack for aligning the start
    void* base = mmap(nullptr, map_len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (base == MAP_FAILED) return set_error(IPG_ENOMEM, "ipg_host_alloc: mmap of %zu bytes failed", map_len);
    const uintptr_t b = (uintptr_t)base;
    const uintptr_t a = (b + granule - 1) / granule * granule;
    if (a > b) munmap(base, a - b);
    if (b + map_len > a + len) munmap((void*)(a + len), b + map_len - (a + len));
    void* p = (void*)a;
    if (granule > page) {
        madvise(p, len, MADV_HUGEPAGE);  // advice only: ignored where the kernel has no THP
        // first touch with one write per huge page, so each fault can take a whole huge page
        for (size_t off = 0; off < len; off += granule) static_cast<volatile char*>(p)[off] = 0;
        madvise(p, len, MADV_COLLAPSE);  // best effort; an error leaves the pages as they are
    }
    cudaError_t e = cudaHostRegister(p, len, cudaHostRegisterPortable);
    if (e != cudaSuccess) {
        cudaGetLastError();
        munmap(p, len);
        return set_error(e == cudaErrorMemoryAllocation ? IPG_ENOMEM : IPG_ECUDA,
                         "ipg_host_alloc: cudaHostRegister of %zu bytes failed: %s", len, cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        host_blocks()[p] = HostBlock{p, len};
    }
    *out = p;
    return IPG_OK;
}

extern "C" ipg_status ipg_host_free(void* p) {
    if (!p) return IPG_OK;
    HostBlock blk;
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        auto it = host_blocks().find(p);
        if (it == host_blocks().end())
            return set_error(IPG_EINVAL, "ipg_host_free: %p did not come from ipg_host_alloc", p);
        blk = it->second;
        host_blocks().erase(it);
    }
    cudaError_t e = cudaHostUnregister(blk.map);
    if (e != cudaSuccess) cudaGetLastError();
    munmap(blk.map, blk.len);
    if (e != cudaSuccess && e != cudaErrorCudartUnloading)
        return set_error(IPG_ECUDA, "ipg_host_free: cudaHostUnregister failed: %s", cudaGetErrorString(e));
    return IPG_OK;
}
