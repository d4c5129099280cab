// Index-checked builds.  Compiled with -DDNS_CHECKED (the library
// libdns_checked.so, built on request), every global-memory load and store
// of the DNS kernels, and the source range of every bulk copy, is first
// compared with the device table of the address ranges the handle owns (its
// device buffers without their guard regions, plus the caller's device
// buffers of the call in progress).  An access outside all of them is not
// made: a load yields zero, a store and a copy are skipped, and the first
// such access records kErrIndex, the source line and the address in the
// handle's device status word, which dns_synchronize reports as
// DNS_ERR_INDEX.  Without -DDNS_CHECKED the macros are the plain accesses.
//
// The table is [0] the number of ranges n, then n (begin, end) byte
// addresses.  A null table (a context that has none) accepts everything.
#pragma once

namespace dns {

constexpr int kErrIndex = 2;
constexpr int kMaxCheckRanges = 64;

// What a checked access needs: the range table and the status word
// ([0] code, [1] source line, [2..3] the address as 64 bits).
struct Chk {
    const unsigned long long *rng = nullptr;
    int *err = nullptr;
};

#ifdef DNS_CHECKED
static __device__ __noinline__ bool addr_ok(const unsigned long long *rng, int *err, const void *p,
                                            unsigned long long bytes, int line) {
    if (!rng) return true;
    const unsigned long long a = (unsigned long long)p, b = a + bytes;
    const unsigned long long n = rng[0];
    for (unsigned long long i = 0; i < n; ++i)
        if (a >= rng[1 + 2 * i] && b <= rng[2 + 2 * i]) return true;
    if (err && atomicCAS(err, 0, kErrIndex) == 0) {
        err[1] = line;
        *reinterpret_cast<unsigned long long *>(err + 2) = a;
        __threadfence();
    }
    return false;
}

template <typename T>
__device__ __forceinline__ T chk_ld(const unsigned long long *rng, int *err, const T *p, int line) {
    if (!addr_ok(rng, err, p, sizeof(T), line)) return T{};
    return *p;
}

template <typename T>
__device__ __forceinline__ void chk_st(const unsigned long long *rng, int *err, T *p, const T &v, int line) {
    if (addr_ok(rng, err, p, sizeof(T), line)) *p = v;
}

#define DNS_LD(c, p) ::dns::chk_ld((c).rng, (c).err, (p), __LINE__)
#define DNS_ST(c, p, v) ::dns::chk_st((c).rng, (c).err, (p), (v), __LINE__)
#define DNS_RANGE_OK(c, p, bytes) \
    ::dns::addr_ok((c).rng, (c).err, (const void *)(p), (unsigned long long)(bytes), __LINE__)
#else
#define DNS_LD(c, p) (*(p))
#define DNS_ST(c, p, v) (void)(*(p) = (v))
#define DNS_RANGE_OK(c, p, bytes) true
#endif

}  // namespace dns
