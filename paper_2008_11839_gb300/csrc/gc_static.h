// gc_static.h -- internal interfaces between the static, BFS, rounds and
// incremental translation units.
#pragma once
#include "gc_internal.h"
#include "uf_device.cuh"

namespace gc {

void uf_triple(const Variant& v, int* L, int* F, int* S);
// Finishes that run in synchronous rounds (a device-side loop).
inline bool is_rounds_link(int link) {
    return link == GCONN_LINK_SV || link == GCONN_LINK_LT || link == GCONN_LINK_LP || link == GCONN_LINK_STERGIOU;
}
UFState make_state(uint32_t n, uint32_t* P, uint32_t* H, u64w* W, uint32_t* sf, const Variant& v);
gconn_status init_state(const UFState& s, cudaStream_t st, uint32_t* zero = nullptr, uint32_t nzero = 0);
gconn_status union_coo(const Variant& v, const UFState& s, const uint32_t* edges, uint64_t m, uint32_t eid_base,
                       cudaStream_t st);
gconn_status compress_all(const Variant& v, const UFState& s, cudaStream_t st);
gconn_status finalize_labels(const Variant& v, const UFState& s, uint32_t* labels, cudaStream_t st);
gconn_status sf_output(uint32_t n, const uint32_t* sf, uint64_t* forest, uint64_t* count, cudaStream_t st);

// BFS sampling (Algorithm 4): labels the source's component with its minimum
// id (in P, or in W for Union-JTB), records BFS-tree arcs in s.sf, and writes
// that minimum as L_max.
// Instantiated for uint32_t and uint64_t CSR offsets.
template <class OffT>
gconn_status bfs_sample(const Variant& v, const UFState& s, const OffT* off, const uint32_t* cols,
                        uint32_t* lmax_dev, cudaStream_t st);

// Round-based finishes (Shiloach-Vishkin, Liu-Tarjan, label propagation,
// Stergiou) over a COO list with optional per-edge forest ids (NULL = the
// edge index).  P ends fully
// compressed and min-rooted.  *edge_passes (optional) receives the number of
// kernel passes that read the whole edge list.
// With m_dev set, the edge count is read on the device (min(*m_dev, m)).
// Each finish is one cooperative launch that loops over its rounds on the
// device; only a non-null edge_passes makes the host wait for the count.
gconn_status rounds_coo(const Variant& v, const UFState& s, const uint32_t* edges, const uint32_t* eids,
                        uint64_t m, cudaStream_t st, uint32_t* edge_passes = nullptr,
                        const unsigned long long* m_dev = nullptr);

// The same over the arcs of the active CSR vertices gathered by k_vg.
template <class OffT>
gconn_status rounds_csr(const Variant& v, const UFState& s, const OffT* off, const uint32_t* cols,
                        const uint32_t* active, const uint32_t* small, const uint32_t* nsmall,
                        const unsigned long long* tasks, const uint32_t* ntasks, uint32_t task_cap,
                        const uint32_t* over, const uint32_t* nover, cudaStream_t st);

}  // namespace gc
