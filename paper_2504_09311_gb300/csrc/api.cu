// api.cu -- error reporting, version, and the batched entry point.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <string>

#include <chrono>

#include "dupin_internal.h"

static thread_local std::string t_last_error;

void dupin_set_error(const std::string &msg) { t_last_error = msg; }

int dupin_fail(int code, const std::string &msg) {
    t_last_error = msg;
    return code;
}

int dupin_cuda_fail(cudaError_t e, const char *what) {
    t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return DUPIN_ERR_CUDA;
}

extern "C" int dupin_last_error(char *buf, size_t cap) {
    if (!buf || cap == 0) return DUPIN_ERR_INVALID_ARG;
    size_t k = t_last_error.size() < cap - 1 ? t_last_error.size() : cap - 1;
    memcpy(buf, t_last_error.data(), k);
    buf[k] = 0;
    return DUPIN_OK;
}

extern "C" const char *dupin_version(void) { return "0.3.0"; }

extern "C" int64_t dupin_struct_size(const char *name) {
    if (!name) return -1;
    const std::string n(name);
    if (n == "dupin_graph_desc") return (int64_t)sizeof(dupin_graph_desc);
    if (n == "dupin_params") return (int64_t)sizeof(dupin_params);
    if (n == "dupin_result") return (int64_t)sizeof(dupin_result);
    if (n == "dupin_serve_config") return (int64_t)sizeof(dupin_serve_config);
    if (n == "dupin_serve_stats_t") return (int64_t)sizeof(dupin_serve_stats_t);
    return -1;
}

// The key of the arc fingerprints that the symmetry checks sum (sym_mix): one
// per process, drawn at first use from the clock and an address, so that no
// fixed input can be built to cancel a missing reverse arc.
unsigned long long fingerprint_key() {
    static const unsigned long long key = fmix64(
        (unsigned long long)std::chrono::steady_clock::now().time_since_epoch().count() ^
        (unsigned long long)(uintptr_t)&key ^ 0x5bd1e9955bd1e995ULL);
    return key;
}
