// Kernel unit for one mesh size; the build compiles this file once per
// supported N with -DDNS_N=<N>.
#include "dns_launch.cuh"

#ifndef DNS_N
#error "compile with -DDNS_N=<mesh size>"
#endif

#define DNS_CAT2(a, b) a##b
#define DNS_CAT(a, b) DNS_CAT2(a, b)

namespace dns {
bool DNS_CAT(get_passes_, DNS_N)(int dtype, PassSet *ps) { return fill_passes<DNS_N>(dtype, ps); }
}  // namespace dns
