// Applies with the fields in host memory: each right-hand side is copied to the
// device, A (or Q A) is applied, and the result is copied back, with the copies
// of one right-hand side overlapping the apply of the previous one (two device
// slots; host-to-device and device-to-host copies on two streams of their own,
// the applies on the caller's stream).  The operator and its arithmetic are those
// of spm_apply_A / spm_apply_QA; only the data movement differs.
#include "common.cuh"

namespace {

struct Pipe {
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    cudaEvent_t in[2] = {nullptr, nullptr}, comp[2] = {nullptr, nullptr}, out[2] = {nullptr, nullptr};
    ~Pipe()
    {
        if (h2d) cudaStreamSynchronize(h2d);
        if (d2h) cudaStreamSynchronize(d2h);
        for (int k = 0; k < 2; ++k) {
            if (in[k]) cudaEventDestroy(in[k]);
            if (comp[k]) cudaEventDestroy(comp[k]);
            if (out[k]) cudaEventDestroy(out[k]);
        }
        if (start) cudaEventDestroy(start);
        if (done) cudaEventDestroy(done);
        if (h2d) cudaStreamDestroy(h2d);
        if (d2h) cudaStreamDestroy(d2h);
    }
};

spm_status apply_host(spm_problem_s *P, spm_prec prec, bool with_q, const void *xh, void *yh, int nrhs, cudaStream_t s)
{
    const size_t el = prec == SPM_C128 ? 16 : 8;
    const size_t per = el * 3 * (size_t)P->n * P->n * P->n; // bytes of one field
    const int slots = nrhs > 1 ? 2 : 1;
    DevBuf din, dout;
    SPM_TRY(din.ensure(per * slots));
    SPM_TRY(dout.ensure(per * slots));
    if (with_q) SPM_TRY(P->kry.ensure(per > P->kry.bytes ? per : P->kry.bytes));
    Pipe pp;
    SPM_CUDA_TRY(cudaStreamCreateWithFlags(&pp.h2d, cudaStreamNonBlocking));
    SPM_CUDA_TRY(cudaStreamCreateWithFlags(&pp.d2h, cudaStreamNonBlocking));
    SPM_CUDA_TRY(cudaEventCreateWithFlags(&pp.start, cudaEventDisableTiming));
    SPM_CUDA_TRY(cudaEventCreateWithFlags(&pp.done, cudaEventDisableTiming));
    for (int k = 0; k < slots; ++k) {
        SPM_CUDA_TRY(cudaEventCreateWithFlags(&pp.in[k], cudaEventDisableTiming));
        SPM_CUDA_TRY(cudaEventCreateWithFlags(&pp.comp[k], cudaEventDisableTiming));
        SPM_CUDA_TRY(cudaEventCreateWithFlags(&pp.out[k], cudaEventDisableTiming));
    }
    // the copies start after the work already queued on the caller's stream
    SPM_CUDA_TRY(cudaEventRecord(pp.start, s));
    SPM_CUDA_TRY(cudaStreamWaitEvent(pp.h2d, pp.start, 0));
    SPM_CUDA_TRY(cudaStreamWaitEvent(pp.d2h, pp.start, 0));
    const char *x = static_cast<const char *>(xh);
    char *y = static_cast<char *>(yh);
    for (int b = 0; b < nrhs; ++b) {
        const int k = b % slots;
        char *di = din.as<char>() + k * per, *dn = dout.as<char>() + k * per;
        // slot k's input is free once the apply of right-hand side b - 2 has run
        if (b >= slots) SPM_CUDA_TRY(cudaStreamWaitEvent(pp.h2d, pp.comp[k], 0));
        SPM_CUDA_TRY(cudaMemcpyAsync(di, x + (size_t)b * per, per, cudaMemcpyHostToDevice, pp.h2d));
        SPM_CUDA_TRY(cudaEventRecord(pp.in[k], pp.h2d));
        SPM_CUDA_TRY(cudaStreamWaitEvent(s, pp.in[k], 0));
        // slot k's output is free once the copy-out of right-hand side b - 2 has run
        if (b >= slots) SPM_CUDA_TRY(cudaStreamWaitEvent(s, pp.out[k], 0));
        if (with_q) {
            SPM_TRY(spm_apply_A_impl(P, prec, di, P->kry.ptr, 1, s));
            SPM_TRY(spm_apply_Q_impl(P, prec, P->kry.ptr, dn, 1, s));
        } else {
            SPM_TRY(spm_apply_A_impl(P, prec, di, dn, 1, s));
        }
        SPM_CUDA_TRY(cudaEventRecord(pp.comp[k], s));
        SPM_CUDA_TRY(cudaStreamWaitEvent(pp.d2h, pp.comp[k], 0));
        SPM_CUDA_TRY(cudaMemcpyAsync(y + (size_t)b * per, dn, per, cudaMemcpyDeviceToHost, pp.d2h));
        SPM_CUDA_TRY(cudaEventRecord(pp.out[k], pp.d2h));
    }
    // the caller's stream sees the last copy-out; the call returns with y_host filled
    SPM_CUDA_TRY(cudaEventRecord(pp.done, pp.d2h));
    SPM_CUDA_TRY(cudaStreamWaitEvent(s, pp.done, 0));
    SPM_CUDA_TRY(cudaStreamSynchronize(s));
    return SPM_OK;
}

spm_status check_host(spm_problem P, spm_prec prec, const void *x, void *y, int nrhs)
{
    if (!P) { spm_set_error("NULL problem"); return SPM_ERR_INVALID_ARG; }
    if (prec != SPM_C128 && prec != SPM_C64) { spm_set_error("precision must be SPM_C128 or SPM_C64"); return SPM_ERR_INVALID_ARG; }
    if (nrhs < 0 || nrhs > 65535) { spm_set_error("nrhs must be in [0, 65535]"); return SPM_ERR_INVALID_ARG; }
    if (nrhs > 0 && (!x || !y)) { spm_set_error("NULL buffer"); return SPM_ERR_INVALID_ARG; }
    if (nrhs > 0 && x == y) { spm_set_error("input and output alias"); return SPM_ERR_INVALID_ARG; }
    return SPM_OK;
}

} // namespace

extern "C" spm_status spm_apply_A_host(spm_problem P, spm_prec prec, const void *x_host, void *y_host, int nrhs,
                                       void *stream)
{
    SPM_TRY(check_host(P, prec, x_host, y_host, nrhs));
    if (nrhs == 0) return SPM_OK;
    return apply_host(P, prec, false, x_host, y_host, nrhs, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" spm_status spm_apply_QA_host(spm_problem P, spm_prec prec, const void *x_host, void *y_host, int nrhs,
                                        void *stream)
{
    SPM_TRY(check_host(P, prec, x_host, y_host, nrhs));
    if (nrhs == 0) return SPM_OK;
    if (!P->have_stencils) { spm_set_error("stencils not built"); return SPM_ERR_NOT_BUILT; }
    return apply_host(P, prec, true, x_host, y_host, nrhs, reinterpret_cast<cudaStream_t>(stream));
}
