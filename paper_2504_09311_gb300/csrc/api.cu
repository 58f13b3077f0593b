// api.cu -- error reporting, version, and the batched entry point.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <string>

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

extern "C" const char *dupin_version(void) { return "0.1.0"; }
