// host_pipeline.cu -- dense rotation from and to host memory (dmrg_rotate_ops_host).
//
// The operator batch is split into chunks of consecutive operators (operators are
// independent given U, the property the paper's UMD split relies on, Sec. 3.2).
// Four streams overlap the work: chunk c+1 is copied in on the copy-in stream
// while chunk c is rotated and chunk c-1 is copied out on the copy-out stream.
// Rotations alternate between the caller's stream and a second compute stream
// (each with its own workspace), so the last, partly filled wave of one chunk's
// kernels overlaps the next chunk's.  Device staging is double buffered; events
// order every reuse of a buffer.  U is copied once and packed once per workspace.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "api_common.h"

using namespace dmrg;

namespace {

// Chunk boundaries.  chunk > 0: equal chunks of that many operators.  chunk == 0:
// about five equal chunks, but the first and the last are cut to a third, so that
// the copy-in before the first rotation and the copy-out after the last one, which
// nothing overlaps, are short.
std::vector<int64_t> chunk_starts(int64_t K, int64_t chunk) {
    std::vector<int64_t> st;
    if (K <= 0) return st;
    if (chunk > 0) {
        for (int64_t k = 0; k < K; k += chunk) st.push_back(k);
    } else {
        const int64_t base = std::max<int64_t>(1, (K + 4) / 5);
        const int64_t edge = std::max<int64_t>(1, (base + 2) / 3);
        if (K <= 2 * edge) {
            for (int64_t k = 0; k < K; k += edge) st.push_back(k);
        } else {
            // first and last chunks of `edge`, the middle split evenly into chunks <= base
            const int64_t mid = K - 2 * edge, n = (mid + base - 1) / base;
            st.push_back(0);
            for (int64_t i = 0; i < n; ++i) st.push_back(edge + mid * i / n);
            st.push_back(K - edge);
        }
    }
    st.push_back(K);
    return st;
}

struct HostDims {
    int64_t chunk, nchunks;   // largest chunk, number of chunks
    std::vector<int64_t> starts;
    size_t es_in, es_out;
    WsLayout ws;   // U, O[2], Oout[2], rotation workspace for one chunk
};

HostDims host_dims(int64_t K, int64_t m, int d, int64_t mp, dmrg_precision p, int in_is_fp64,
                   int64_t chunk) {
    HostDims H;
    H.starts = chunk_starts(K, chunk);
    H.nchunks = H.starts.empty() ? 0 : int64_t(H.starts.size()) - 1;
    H.chunk = 1;
    for (int64_t c = 0; c < H.nchunks; ++c) H.chunk = std::max(H.chunk, H.starts[c + 1] - H.starts[c]);
    H.es_in = in_is_fp64 ? 8 : 4;
    H.es_out = p == DMRG_PREC_FP64 ? 8 : 4;
    H.ws.add("U", size_t(m) * d * mp * 8);
    H.ws.add("O0", size_t(H.chunk) * m * m * H.es_in);
    H.ws.add("O1", size_t(H.chunk) * m * m * H.es_in);
    H.ws.add("R0", size_t(H.chunk) * mp * mp * H.es_out);
    H.ws.add("R1", size_t(H.chunk) * mp * mp * H.es_out);
    H.ws.add("rot0", dense_dims(H.chunk, m, d, mp, p).ws.total);
    H.ws.add("rot1", dense_dims(H.chunk, m, d, mp, p).ws.total);
    return H;
}

cudaError_t ensure_pipeline(dmrg_handle h) {
    cudaError_t e = cudaSuccess;
    if (!h->copy_in) e = cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !h->copy_out) e = cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking);
    if (e == cudaSuccess && !h->compute2) e = cudaStreamCreateWithFlags(&h->compute2, cudaStreamNonBlocking);
    cudaEvent_t* evs[8] = {&h->ev_start, &h->ev_u, &h->ev_in[0], &h->ev_in[1],
                           &h->ev_comp[0], &h->ev_comp[1], &h->ev_out[0], &h->ev_out[1]};
    for (cudaEvent_t* ev : evs)
        if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    return e;
}

}  // namespace

extern "C" {

dmrg_status dmrg_rotate_ops_host_workspace(dmrg_handle h, int64_t K, int64_t m, int d, int64_t mp,
                                           dmrg_precision p, int in_is_fp64, int64_t chunk,
                                           size_t* bytes) {
    if (!bytes) return fail(h, DMRG_ERR_INVALID_ARG, "bytes is NULL");
    dmrg_status st = check_dense_args(h, K, m, d, mp, p);
    if (st != DMRG_OK) return st;
    *bytes = host_dims(K, m, d, mp, p, in_is_fp64, chunk).ws.total;
    return DMRG_OK;
}

dmrg_status dmrg_rotate_ops_host(dmrg_handle h, const double* U, int64_t m, int d, int64_t mp,
                                 const void* O, int in_is_fp64, int64_t K, void* Oout,
                                 dmrg_precision p, int64_t chunk, void* ws, size_t ws_bytes,
                                 dmrg_stream_t stream) {
    dmrg_status st = check_dense_args(h, K, m, d, mp, p);
    if (st != DMRG_OK) return st;
    if (K == 0) return DMRG_OK;
    if (!U || !O || !Oout) return fail(h, DMRG_ERR_INVALID_ARG, "null data pointer");
    if (p == DMRG_PREC_FP64 && !in_is_fp64)
        return fail(h, DMRG_ERR_INVALID_ARG, "the FP64 precision needs FP64 operators");
    const bool tc = (p == DMRG_PREC_TF32 || p == DMRG_PREC_BF16X3);
    if (tc && !tc_supported(h)) return fail(h, DMRG_ERR_UNSUPPORTED, "tensor cores need sm_103");
    const HostDims H = host_dims(K, m, d, mp, p, in_is_fp64, chunk);
    st = check_ws(h, ws, ws_bytes, H.ws.total);
    if (st != DMRG_OK) return st;
    cudaError_t e = ensure_pipeline(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "pipeline streams");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(ws);
    double* Ud = reinterpret_cast<double*>(base + H.ws.offsets[0]);
    void* Od[2] = {base + H.ws.offsets[1], base + H.ws.offsets[2]};
    void* Rd[2] = {base + H.ws.offsets[3], base + H.ws.offsets[4]};
    void* rot[2] = {base + H.ws.offsets[5], base + H.ws.offsets[6]};
    cudaStream_t cs[2] = {s, h->compute2};
    const size_t op_in = size_t(m) * m * H.es_in, op_out = size_t(mp) * mp * H.es_out;
    const TcMode mode = (p == DMRG_PREC_BF16X3) ? TC_BF16X3 : TC_TF32;

    // everything the caller queued before this call happens first
    if ((e = cudaEventRecord(h->ev_start, s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(h->copy_in, h->ev_start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(h->copy_out, h->ev_start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(h->compute2, h->ev_start, 0)) != cudaSuccess)
        return cuda_fail(h, e, "ordering");
    e = cudaMemcpyAsync(Ud, U, size_t(m) * d * mp * 8, cudaMemcpyHostToDevice, h->copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_u, h->copy_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_u, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->compute2, h->ev_u, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy U");
    for (int64_t c = 0; c < H.nchunks; ++c) {
        const int b = int(c & 1);
        const int64_t k0 = H.starts[c], kc = H.starts[c + 1] - k0;
        // copy in: the buffer is free once the rotation of chunk c-2 has read it
        if (c >= 2 && (e = cudaStreamWaitEvent(h->copy_in, h->ev_comp[b], 0)) != cudaSuccess)
            return cuda_fail(h, e, "ordering");
        e = cudaMemcpyAsync(Od[b], static_cast<const char*>(O) + size_t(k0) * op_in, size_t(kc) * op_in,
                            cudaMemcpyHostToDevice, h->copy_in);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[b], h->copy_in);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy in");
        // rotate on compute stream b: inputs landed, and the output buffer was copied out
        // (chunk c-2, which ran on the same stream)
        cudaStream_t x = cs[b];
        if ((e = cudaStreamWaitEvent(x, h->ev_in[b], 0)) != cudaSuccess) return cuda_fail(h, e, "ordering");
        if (c >= 2 && (e = cudaStreamWaitEvent(x, h->ev_out[b], 0)) != cudaSuccess)
            return cuda_fail(h, e, "ordering");
        const TcConfig c1 = tc ? tuned_config(h, shape_key("g1", kc, m, d, mp, p), mode) : TcConfig();
        const TcConfig c2 = tc ? tuned_config(h, shape_key("g2", kc, m, d, mp, p), mode) : TcConfig();
        st = tc ? dense_tc_forward(h, Ud, m, d, mp, Od[b], in_is_fp64, kc, Rd[b], p, rot[b], c1, c2, x,
                                   c < 2)
                : dense_simt_forward(h, Ud, m, d, mp, Od[b], in_is_fp64, kc, Rd[b], p, rot[b], x, c < 2);
        if (st != DMRG_OK) return st;
        if ((e = cudaEventRecord(h->ev_comp[b], x)) != cudaSuccess) return cuda_fail(h, e, "ordering");
        // copy out
        if ((e = cudaStreamWaitEvent(h->copy_out, h->ev_comp[b], 0)) != cudaSuccess)
            return cuda_fail(h, e, "ordering");
        e = cudaMemcpyAsync(static_cast<char*>(Oout) + size_t(k0) * op_out, Rd[b], size_t(kc) * op_out,
                            cudaMemcpyDeviceToHost, h->copy_out);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_out[b], h->copy_out);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy out");
    }
    // the caller's stream completes only after the last copy out
    for (int b = 0; b < 2 && b < H.nchunks; ++b)
        if ((e = cudaStreamWaitEvent(s, h->ev_out[b], 0)) != cudaSuccess) return cuda_fail(h, e, "ordering");
    return DMRG_OK;
}

}  // extern "C"
