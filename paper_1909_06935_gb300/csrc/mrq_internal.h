// mrq_internal.h - what the runtime (mrq.cu) shares with the other translation units of the
// library: a read-only view of a context's loaded Hamiltonian and its error slot.  Not part of
// the C ABI.
#ifndef MRQ_INTERNAL_H
#define MRQ_INTERNAL_H

#include <cuda_runtime.h>

struct mrq_ctx;

struct MrqHamView {
    int device;
    cudaStream_t stream;
    int n, nc, na, nv, nalpha, nbeta, W;
    const double* h1;        // n x n row-major, device
    const double* eri;       // 8-fold packed (pq|rs), device
    long long neri;
    double e_nuc;
};

// MRQ_NOT_LOADED (message set) when the context holds no Hamiltonian
int mrq_internal_ham(mrq_ctx* ctx, MrqHamView* out);
// record a message in the context's error slot and return code
int mrq_internal_fail(mrq_ctx* ctx, int code, const char* fmt, ...);
// the context's host-wait (deadline-aware) synchronisation
int mrq_internal_sync(mrq_ctx* ctx);

#endif
