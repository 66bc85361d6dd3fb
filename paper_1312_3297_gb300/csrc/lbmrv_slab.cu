// Slab decomposition of a periodic lattice (declarations and contracts in include/lbmrv.h).
//
// What is split is the exact transport of Section 1.1 (relation (transport)): in pull form
// a node reads population j from x - v_j dt, so a layer (a row of a D2Q9 lattice, a z-plane
// of a D3Q19 lattice) needs, from each neighbouring layer, only the populations whose
// velocity crosses between them: 3 of 9 for D2Q9 (c_y = +-1), 5 of 19 for D3Q19 (c_z = +-1).
// A slab handle holds its own layers plus one halo layer on each side. Before each step the
// edge layers' crossing populations are packed into contiguous buffers, exchanged with the
// neighbouring slabs (by the caller: a peer copy, NCCL or any transport), and unpacked into
// the halo layers. The step then runs unchanged over the whole slab; what it computes in the
// halo layers is never read, since the next exchange overwrites every halo value a step reads.
//
// Buffer order (shared by the host index maps and the device kernels): value b of a face
// buffer is crossing population k = b / L (in ascending population index) at in-layer node
// i = b % L, L the layer size.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "handle.h"
#include "launch.h"
#include "lbmrv.h"
#include "pdl.cuh"

using namespace lbmrv;

namespace {

// Component of each velocity along the slab axis (y for D2Q9, z for D3Q19), in the
// population order of include/lbmrv.h.
constexpr int kAxisD2Q9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
constexpr int kAxisD3Q19[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

struct Crossing {
    int count = 0;
    int j[5] = {0, 0, 0, 0, 0};
};

// Populations whose velocity has axis component `sign` (+1 or -1), ascending.
Crossing crossing(int lattice, int sign) {
    Crossing c;
    const bool d3 = lattice == LBMRV_D3Q19;
    const int q = d3 ? 19 : 9;
    for (int j = 0; j < q; ++j)
        if ((d3 ? kAxisD3Q19[j] : kAxisD2Q9[j]) == sign) c.j[c.count++] = j;
    return c;
}

// Layer size and count of a slab lattice; false when the dims are not a valid slab (at
// least one interior layer between the two halo layers).
bool slab_shape(int lattice, const int64_t dims[3], int64_t* L, int64_t* m, int64_t* n) {
    if (!dims || dims[0] < 1 || dims[1] < 1) return false;
    if (lattice == LBMRV_D3Q19) {
        if (dims[2] < 3) return false;
        *L = dims[0] * dims[1];
        *m = dims[2];
    } else if (lattice == LBMRV_D2Q9 || lattice == LBMRV_D2Q9_CASCADED) {
        if (dims[1] < 3 || (dims[2] != 1 && dims[2] != 0)) return false;
        *L = dims[0];
        *m = dims[1];
    } else {
        return false;
    }
    *n = *L * *m;
    return *n < (int64_t(1) << 31);
}

// Which layer and populations one face transfers. side 0 is the lower face, side 1 the
// upper face. Sent: the edge interior layer's populations moving across the face (down,
// c = -1, through the lower face; up, c = +1, through the upper face). Received: the halo
// layer's populations moving in from across the face (c = +1 into layer 0, c = -1 into
// layer m - 1).
struct Face {
    int64_t layer;
    Crossing pops;
};
Face send_face(int lattice, int64_t m, int side) {
    return side == 0 ? Face{1, crossing(lattice, -1)} : Face{m - 2, crossing(lattice, +1)};
}
Face recv_face(int lattice, int64_t m, int side) {
    return side == 0 ? Face{0, crossing(lattice, +1)} : Face{m - 1, crossing(lattice, -1)};
}

// The adjoint exchange runs the other way. The reverse step gathers mu_{k+1}(x + c_j) (the
// transpose of the pull), so an edge layer needs from the halo layer beyond it the
// populations whose velocity points out through that face: the lower face sends layer 1's
// c = +1 populations and receives c = -1 populations into layer 0; the upper face sends
// layer m-2's c = -1 populations and receives c = +1 populations into layer m-1.
Face send_face_adjoint(int lattice, int64_t m, int side) {
    return side == 0 ? Face{1, crossing(lattice, +1)} : Face{m - 2, crossing(lattice, -1)};
}
Face recv_face_adjoint(int lattice, int64_t m, int side) {
    return side == 0 ? Face{0, crossing(lattice, -1)} : Face{m - 1, crossing(lattice, +1)};
}

// Copies between the two face buffers and the state, value b of face f (blockIdx.y) <->
// state[j_k n + layer L + i]. PACK: buffers <- state; otherwise state <- buffers. E: an
// unsigned type of the storage element's size (the values are moved as bits). A NULL
// buffer skips its face. Launched as a dependent launch: it waits for the work before it in
// the stream (the step that wrote the state, or the copy that filled the buffers) before
// touching memory.
template <typename E, bool PACK>
__global__ void k_halo_copy(E* __restrict__ state, E* __restrict__ buf_lo,
                            E* __restrict__ buf_hi, int64_t n, int64_t L, Face lo, Face hi) {
    pdl_wait_prior();
    pdl_allow_next();
    const Face& f = blockIdx.y == 0 ? lo : hi;
    E* __restrict__ buf = blockIdx.y == 0 ? buf_lo : buf_hi;
    if (!buf) return;
    const int64_t total = (int64_t)f.pops.count * L;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < total;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(b / L);
        const int64_t i = b - (int64_t)k * L;
        const int64_t off = (int64_t)f.pops.j[k] * n + f.layer * L + i;
        if (PACK)
            buf[b] = state[off];
        else
            state[off] = buf[b];
    }
}

// Both faces in one launch (grid y = face), between `state` (elements of `elem` bytes, the
// handle's layout) and the two buffers.
template <bool PACK>
cudaError_t halo_copy(const lbmrv_s* h, void* state, int64_t elem, void* buf_lo,
                      void* buf_hi, const Face& lo, const Face& hi) {
    const int64_t L = layer_size(h), total = (int64_t)lo.pops.count * L;
    const dim3 grid((unsigned)grid_stride_blocks(total, 256), 2);
    if (elem == 4)
        return launch_pdl(k_halo_copy<uint32_t, PACK>, grid, dim3(256), h->stream,
                          static_cast<uint32_t*>(state), static_cast<uint32_t*>(buf_lo),
                          static_cast<uint32_t*>(buf_hi), h->n, L, lo, hi);
    return launch_pdl(k_halo_copy<uint16_t, PACK>, grid, dim3(256), h->stream,
                      static_cast<uint16_t*>(state), static_cast<uint16_t*>(buf_lo),
                      static_cast<uint16_t*>(buf_hi), h->n, L, lo, hi);
}

}  // namespace

extern "C" {

int lbmrv_slab_plan(int64_t extent, int ranks, int rank, int64_t* first, int64_t* count) {
    if (!first || !count || ranks < 1 || rank < 0 || rank >= ranks || extent < ranks)
        return LBMRV_E_INVAL;
    const int64_t base = extent / ranks, extra = extent % ranks;
    *count = base + (rank < extra ? 1 : 0);
    *first = (int64_t)rank * base + (rank < extra ? rank : extra);
    return LBMRV_OK;
}

int64_t lbmrv_halo_count(int lattice, const int64_t dims[3]) {
    int64_t L, m, n;
    if (!slab_shape(lattice, dims, &L, &m, &n)) return -1;
    return (int64_t)crossing(lattice, +1).count * L;
}

int lbmrv_halo_map(int lattice, const int64_t dims[3], int side, int64_t* send_idx,
                   int64_t* recv_idx) {
    int64_t L, m, n;
    if (!slab_shape(lattice, dims, &L, &m, &n) || (side != 0 && side != 1))
        return LBMRV_E_INVAL;
    const Face fs = send_face(lattice, m, side), fr = recv_face(lattice, m, side);
    for (int k = 0; k < fs.pops.count; ++k)
        for (int64_t i = 0; i < L; ++i) {
            if (send_idx) send_idx[k * L + i] = (int64_t)fs.pops.j[k] * n + fs.layer * L + i;
            if (recv_idx) recv_idx[k * L + i] = (int64_t)fr.pops.j[k] * n + fr.layer * L + i;
        }
    return LBMRV_OK;
}

int lbmrv_set_slab(lbmrv_t h, int64_t first, int64_t extent) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_set_slab: NULL handle");
    const int64_t dims[3] = {h->nx, h->ny, h->nz};
    int64_t L, m, n;
    if (!slab_shape(h->lattice, dims, &L, &m, &n))
        return fail(h, LBMRV_E_INVAL, "lbmrv_set_slab: a slab needs at least 3 layers");
    if (extent < m - 2 || first < 0 || first >= extent || extent > (int64_t(1) << 30))
        return fail(h, LBMRV_E_INVAL,
                    "lbmrv_set_slab: need 0 <= first < extent and extent >= %lld layers",
                    (long long)(m - 2));
    h->slab = true;
    h->slab_first = first;
    h->slab_extent = extent;
    h->ref_auto = false;  // every slab must store relative to one shared reference
    return LBMRV_OK;
}

int lbmrv_halo_pack(lbmrv_t h, void* send_lo_dev, void* send_hi_dev) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_halo_pack: NULL handle");
    if (!h->slab) return fail(h, LBMRV_E_INVAL, "lbmrv_halo_pack: not a slab (lbmrv_set_slab)");
    DeviceGuard g(h->device);
    const int64_t m = layer_count(h);
    if (!send_lo_dev && !send_hi_dev) return LBMRV_OK;
    const cudaError_t e = halo_copy<true>(h, h->f[h->cur], elem_size(h->storage), send_lo_dev,
                                          send_hi_dev, send_face(h->lattice, m, 0),
                                          send_face(h->lattice, m, 1));
    return e == cudaSuccess ? LBMRV_OK : cuda_fail(h, e, "lbmrv_halo_pack");
}

int lbmrv_halo_unpack(lbmrv_t h, const void* recv_lo_dev, const void* recv_hi_dev) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_halo_unpack: NULL handle");
    if (!h->slab)
        return fail(h, LBMRV_E_INVAL, "lbmrv_halo_unpack: not a slab (lbmrv_set_slab)");
    DeviceGuard g(h->device);
    const int64_t m = layer_count(h);
    if (!recv_lo_dev && !recv_hi_dev) return LBMRV_OK;
    const cudaError_t e = halo_copy<false>(h, h->f[h->cur], elem_size(h->storage),
                                           const_cast<void*>(recv_lo_dev),
                                           const_cast<void*>(recv_hi_dev),
                                           recv_face(h->lattice, m, 0),
                                           recv_face(h->lattice, m, 1));
    return e == cudaSuccess ? LBMRV_OK : cuda_fail(h, e, "lbmrv_halo_unpack");
}

int lbmrv_halo_map_adjoint(int lattice, const int64_t dims[3], int side, int64_t* send_idx,
                           int64_t* recv_idx) {
    int64_t L, m, n;
    if (!slab_shape(lattice, dims, &L, &m, &n) || (side != 0 && side != 1))
        return LBMRV_E_INVAL;
    const Face fs = send_face_adjoint(lattice, m, side), fr = recv_face_adjoint(lattice, m, side);
    for (int k = 0; k < fs.pops.count; ++k)
        for (int64_t i = 0; i < L; ++i) {
            if (send_idx) send_idx[k * L + i] = (int64_t)fs.pops.j[k] * n + fs.layer * L + i;
            if (recv_idx) recv_idx[k * L + i] = (int64_t)fr.pops.j[k] * n + fr.layer * L + i;
        }
    return LBMRV_OK;
}

int lbmrv_halo_pack_adjoint(lbmrv_t h, const float* mu_dev, float* send_lo_dev,
                            float* send_hi_dev) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_halo_pack_adjoint: NULL handle");
    if (!h->slab || !mu_dev)
        return fail(h, LBMRV_E_INVAL, "lbmrv_halo_pack_adjoint: not a slab, or NULL mu");
    if (!send_lo_dev && !send_hi_dev) return LBMRV_OK;
    DeviceGuard g(h->device);
    const int64_t m = layer_count(h);
    const cudaError_t e = halo_copy<true>(h, const_cast<float*>(mu_dev), 4, send_lo_dev,
                                          send_hi_dev, send_face_adjoint(h->lattice, m, 0),
                                          send_face_adjoint(h->lattice, m, 1));
    return e == cudaSuccess ? LBMRV_OK : cuda_fail(h, e, "lbmrv_halo_pack_adjoint");
}

int lbmrv_halo_unpack_adjoint(lbmrv_t h, float* mu_dev, const float* recv_lo_dev,
                              const float* recv_hi_dev) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_halo_unpack_adjoint: NULL handle");
    if (!h->slab || !mu_dev)
        return fail(h, LBMRV_E_INVAL, "lbmrv_halo_unpack_adjoint: not a slab, or NULL mu");
    if (!recv_lo_dev && !recv_hi_dev) return LBMRV_OK;
    DeviceGuard g(h->device);
    const int64_t m = layer_count(h);
    const cudaError_t e = halo_copy<false>(h, mu_dev, 4, const_cast<float*>(recv_lo_dev),
                                           const_cast<float*>(recv_hi_dev),
                                           recv_face_adjoint(h->lattice, m, 0),
                                           recv_face_adjoint(h->lattice, m, 1));
    return e == cudaSuccess ? LBMRV_OK : cuda_fail(h, e, "lbmrv_halo_unpack_adjoint");
}

int lbmrv_flow_sums(lbmrv_t h, const float* rho_dev, const float* u_dev, double out_host[4]) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_flow_sums: NULL handle");
    if (!u_dev || !out_host) return fail(h, LBMRV_E_INVAL, "lbmrv_flow_sums: NULL argument");
    DeviceGuard g(h->device);
    const int64_t o = owned_first(h);
    double* res = h->red + 8 * (size_t)h->red_blocks;
    double sums[4] = {0.0, 0.0, 0.0, 0.0};
    cudaError_t e = launch_mean_flow(rho_dev ? rho_dev + o : nullptr, u_dev + o, owned_count(h),
                                     h->n, h->dim, h->red, h->red_blocks, res, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sums, res, sizeof(sums), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_flow_sums");
    for (int c = 0; c < 4; ++c) out_host[c] = sums[c];
    return LBMRV_OK;
}

int lbmrv_set_reference_sums(lbmrv_t h, double rho_ref, const double sums[4]) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_set_reference_sums: NULL handle");
    if (!sums) return fail(h, LBMRV_E_INVAL, "lbmrv_set_reference_sums: NULL sums");
    for (int c = 0; c < 4; ++c)
        if (!std::isfinite(sums[c]))
            return fail(h, LBMRV_E_NONFINITE, "lbmrv_set_reference_sums: non-finite sums");
    if (!(sums[0] > 0.0))
        return fail(h, LBMRV_E_INVAL, "lbmrv_set_reference_sums: the total mass must be positive");
    double u[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < h->dim; ++a) u[a] = sums[1 + a] / sums[0];
    return lbmrv_set_reference(h, rho_ref, u);
}

}  // extern "C"
