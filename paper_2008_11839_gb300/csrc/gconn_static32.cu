// gconn_static32.cu -- static connected components and spanning forest over a
// CSR with uint32_t offsets (graphs with fewer than 2^32 arcs): the same pass
// as gconn_cc_csr / gconn_spanning_forest_csr, reading half the offset bytes
// (Algorithms 1 and 2, Section 3.2; the CSR format of Section 2).
#include "csr_impl.cuh"

using namespace gc;

extern "C" gconn_status gconn_cc_csr32(uint32_t n, const uint32_t* offsets, const uint32_t* cols, uint32_t* labels,
                                       const gconn_variant* v, void* stream) {
    if (!offsets) return GCONN_E_INVAL;
    return static_run<uint32_t>(n, 0, nullptr, offsets, cols, labels, nullptr, nullptr, v, 0, stream);
}

extern "C" gconn_status gconn_spanning_forest_csr32(uint32_t n, const uint32_t* offsets, const uint32_t* cols,
                                                    uint64_t* forest, uint64_t* forest_count, uint32_t* labels,
                                                    const gconn_variant* v, void* stream) {
    if (!offsets) return GCONN_E_INVAL;
    return static_run<uint32_t>(n, 0, nullptr, offsets, cols, labels, forest, forest_count, v, 1, stream);
}
