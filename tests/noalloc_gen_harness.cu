// Test-only build of the no-allocation entry point with a hook that presets
// its merge-table generation, so that a test can make the 32-bit counter wrap
// on its next call.  It includes the library's own source file and is linked
// with the library's other objects into a separate shared library; the
// product library exports no such hook.
#include <cstddef>

#include "itpp_noalloc.cu"

extern "C" int itpp_test_noalloc_set_generation(unsigned int g) {
    return cudaMemcpyToSymbol(g_noalloc_scratch, &g, sizeof g, offsetof(itpp::DevCtl, gen)) ==
                   cudaSuccess
               ? 0
               : 1;
}
