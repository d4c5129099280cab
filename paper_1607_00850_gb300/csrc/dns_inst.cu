// Kernel unit for one mesh size; the build compiles this file once per
// supported N with -DDNS_N=<N> (with -DDNS_STUB: an empty entry).
#include "dns_launch.cuh"

#ifndef DNS_N
#error "compile with -DDNS_N=<mesh size>"
#endif

#define DNS_CAT2(a, b) a##b
#define DNS_CAT(a, b) DNS_CAT2(a, b)

namespace dns {
#ifdef DNS_STUB
// a mesh size left out of this library (the index-checked build compiles a
// subset): no kernels, dns_init reports DNS_ERR_UNSUPPORTED
bool DNS_CAT(get_passes_, DNS_N)(int, PassSet *) { return false; }
#else
bool DNS_CAT(get_passes_, DNS_N)(int dtype, PassSet *ps) { return fill_passes<DNS_N>(dtype, ps); }
#endif
}  // namespace dns
