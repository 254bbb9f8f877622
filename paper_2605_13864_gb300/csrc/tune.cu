// tune.cu -- the autotuner: enumerate the compiled kernel configurations,
// time each one on library-owned scratch buffers with CUDA events, select the
// fastest, and persist the choices in a small text cache.
//
// Cache format, one choice per line:
//   transpose <element bytes> <configuration name>
//   reduce <configuration name>
//   param <name> <integer value>
// Names rather than indices are stored, so a cache survives a rebuild that
// reorders the configuration tables.  OPTIGPU_TUNE_CACHE, if set when the
// library is loaded, names a cache to read.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

namespace optigpu {
namespace {

std::mutex g_tune_mu;

bool op_dtype_ok(int op, int dtype)
{
    return op == OPTIGPU_OP_BATCH || op == OPTIGPU_OP_SCAN ||
           ((op == OPTIGPU_OP_TRANSPOSE || op == OPTIGPU_OP_REDUCE) && dtype_valid(dtype));
}

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events()
    {
        if (a)
            cudaEventDestroy(a);
        if (b)
            cudaEventDestroy(b);
    }
};

struct Scratch {
    void *p = nullptr;
    ~Scratch()
    {
        if (p)
            cudaFree(p);
    }
};

// Median time in ms of `reps` launches of `launch` (after 2 warm-up runs).
template <typename F>
optigpu_status time_median(F launch, int reps, cudaStream_t stream, float &ms)
{
    Events ev;
    optigpu_status st;
    if ((st = check_cuda(cudaEventCreate(&ev.a), "cudaEventCreate")) != OPTIGPU_OK)
        return st;
    if ((st = check_cuda(cudaEventCreate(&ev.b), "cudaEventCreate")) != OPTIGPU_OK)
        return st;
    for (int i = 0; i < 2; ++i)
        if ((st = launch()) != OPTIGPU_OK)
            return st;
    std::vector<float> t;
    for (int i = 0; i < reps; ++i) {
        cudaEventRecord(ev.a, stream);
        if ((st = launch()) != OPTIGPU_OK)
            return st;
        cudaEventRecord(ev.b, stream);
        if ((st = check_cuda(cudaEventSynchronize(ev.b), "cudaEventSynchronize")) != OPTIGPU_OK)
            return st;
        float x = 0.f;
        cudaEventElapsedTime(&x, ev.a, ev.b);
        t.push_back(x);
    }
    std::sort(t.begin(), t.end());
    ms = t[t.size() / 2];
    return OPTIGPU_OK;
}

void load_cache_from_env()
{
    const char *path = std::getenv("OPTIGPU_TUNE_CACHE");
    if (path && *path)
        optigpu_tune_load(path);
}

struct EnvLoader {
    EnvLoader() { load_cache_from_env(); }
} g_env_loader;

} // namespace
} // namespace optigpu

using namespace optigpu;

extern "C" {

int optigpu_tune_num_configs(optigpu_op op, optigpu_dtype dtype)
{
    if (!op_dtype_ok(op, dtype))
        return -1;
    if (op == OPTIGPU_OP_BATCH)
        return batch_num_configs();
    if (op == OPTIGPU_OP_SCAN)
        return scan_num_configs();
    return op == OPTIGPU_OP_TRANSPOSE ? transpose_num_configs(esize_of(dtype)) : reduce_num_configs();
}

const char *optigpu_tune_config_name(optigpu_op op, optigpu_dtype dtype, int config)
{
    if (!op_dtype_ok(op, dtype))
        return nullptr;
    if (op == OPTIGPU_OP_BATCH)
        return batch_config_name(config);
    if (op == OPTIGPU_OP_SCAN)
        return scan_config_name(config);
    return op == OPTIGPU_OP_TRANSPOSE ? transpose_config_name(esize_of(dtype), config) : reduce_config_name(config);
}

optigpu_status optigpu_tune_select(optigpu_op op, optigpu_dtype dtype, int config)
{
    if (!op_dtype_ok(op, dtype))
        return fail(OPTIGPU_ERR_INVALID_ARG, "tune: unknown op or dtype");
    if (config < 0 || config >= optigpu_tune_num_configs(op, dtype))
        return fail(OPTIGPU_ERR_INVALID_ARG, "tune: configuration index out of range");
    if (op == OPTIGPU_OP_BATCH)
        batch_select(config);
    else if (op == OPTIGPU_OP_SCAN)
        scan_select(int(dtype), config);
    else if (op == OPTIGPU_OP_TRANSPOSE)
        transpose_select(esize_of(dtype), config);
    else
        reduce_select(config);
    return OPTIGPU_OK;
}

int optigpu_tune_selected(optigpu_op op, optigpu_dtype dtype)
{
    if (!op_dtype_ok(op, dtype))
        return -1;
    if (op == OPTIGPU_OP_BATCH)
        return batch_selected();
    if (op == OPTIGPU_OP_SCAN)
        return scan_selected(int(dtype));
    return op == OPTIGPU_OP_TRANSPOSE ? transpose_selected(esize_of(dtype)) : reduce_selected();
}

optigpu_status optigpu_tune_set_param(const char *name, int64_t value)
{
    if (!name)
        return fail(OPTIGPU_ERR_INVALID_ARG, "tune: null parameter name");
    if (std::strcmp(name, "transpose.group_rows") == 0) {
        if (value < 1 || value > 4096)
            return fail(OPTIGPU_ERR_INVALID_ARG, "tune: transpose.group_rows must be in [1, 4096]");
        transpose_set_group_rows(int(value));
        return OPTIGPU_OK;
    }
    return fail(OPTIGPU_ERR_NOT_FOUND, std::string("tune: unknown parameter ") + name);
}

int64_t optigpu_tune_get_param(const char *name)
{
    if (name && std::strcmp(name, "transpose.group_rows") == 0)
        return transpose_group_rows();
    return -1;
}

optigpu_status optigpu_autotune(optigpu_op op, optigpu_dtype dtype, int64_t rows, int64_t cols, int reps,
                                optigpu_stream_t stream, int *best_config, float *best_ms)
{
    optigpu::NvtxRange nvtx_range("optigpu_autotune");
    if (!op_dtype_ok(op, dtype) || op == OPTIGPU_OP_BATCH || !dtype_valid(int(dtype)))
        return fail(OPTIGPU_ERR_INVALID_ARG, "autotune: unknown op or dtype (batches: optigpu_batch_autotune)");
    if (rows <= 0 || cols <= 0 || rows > (int64_t(1) << 31) || cols > (int64_t(1) << 31) || reps < 1 ||
        reps > 1000)
        return fail(OPTIGPU_ERR_INVALID_ARG, "autotune: rows, cols in [1, 2^31], reps in [1, 1000]");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t es = esize_of(dtype);
    const size_t bytes = size_t(rows) * size_t(cols) * es;
    Scratch a, b;
    optigpu_status st;
    if ((st = check_cuda(cudaMalloc(&a.p, bytes), "autotune: cudaMalloc")) != OPTIGPU_OK)
        return st;
    if ((st = check_cuda(cudaMemsetAsync(a.p, 0, bytes, s), "autotune: cudaMemsetAsync")) != OPTIGPU_OK)
        return st;
    if (op == OPTIGPU_OP_TRANSPOSE &&
        (st = check_cuda(cudaMalloc(&b.p, bytes), "autotune: cudaMalloc")) != OPTIGPU_OK)
        return st;
    double *out = nullptr;
    if (op == OPTIGPU_OP_REDUCE &&
        (st = check_cuda(cudaMalloc(&b.p, 8), "autotune: cudaMalloc")) != OPTIGPU_OK)
        return st;
    const int64_t n_elems = rows * cols;
    if (op == OPTIGPU_OP_SCAN &&
        (st = check_cuda(cudaMalloc(&b.p, size_t(n_elems) * (dtype == OPTIGPU_INT32 ? 8 : 4)),
                         "autotune: cudaMalloc")) != OPTIGPU_OK)
        return st;
    out = static_cast<double *>(b.p);
    const int n = optigpu_tune_num_configs(op, dtype);
    const int prev = optigpu_tune_selected(op, dtype);
    int best = -1;
    float best_t = 0.f;
    for (int c = 0; c < n; ++c) {
        float ms = 0.f;
        if (op == OPTIGPU_OP_TRANSPOSE) {
            if (c + 1 < n && !optigpu_transpose_tma_eligible(a.p, b.p, rows, cols, dtype))
                continue;
            st = time_median([&] { return transpose_launch_config(a.p, b.p, rows, cols, es, c, s); }, reps, s, ms);
        } else if (op == OPTIGPU_OP_SCAN) {
            scan_select(int(dtype), c);
            st = time_median([&] { return optigpu_scan_inclusive(a.p, b.p, n_elems, dtype, s); }, reps, s, ms);
        } else {
            reduce_select(c);
            st = time_median([&] { return reduce_dispatch(a.p, rows * cols, int(dtype), out, 0u, s); }, reps, s, ms);
        }
        if (st != OPTIGPU_OK) {
            if (op == OPTIGPU_OP_REDUCE)
                reduce_select(prev);
            if (op == OPTIGPU_OP_SCAN)
                scan_select(int(dtype), prev);
            return st;
        }
        if (best < 0 || ms < best_t) {
            best = c;
            best_t = ms;
        }
    }
    if (best < 0)
        return fail(OPTIGPU_ERR_INVALID_ARG, "autotune: no configuration accepts this shape");
    optigpu_tune_select(op, dtype, best);
    if (best_config)
        *best_config = best;
    if (best_ms)
        *best_ms = best_t;
    return OPTIGPU_OK;
}

optigpu_status optigpu_tune_save(const char *path)
{
    if (!path)
        return fail(OPTIGPU_ERR_INVALID_ARG, "tune_save: null path");
    std::ofstream f(path);
    if (!f)
        return fail(OPTIGPU_ERR_INVALID_ARG, std::string("tune_save: cannot open ") + path);
    for (int es : {2, 4}) {
        const optigpu_dtype dt = es == 4 ? OPTIGPU_FLOAT32 : OPTIGPU_BFLOAT16;
        f << "transpose " << es << " " << transpose_config_name(size_t(es), transpose_selected(size_t(es))) << "\n";
        (void)dt;
    }
    f << "reduce " << reduce_config_name(reduce_selected()) << "\n";
    f << "batch " << batch_config_name(batch_selected()) << "\n";
    f << "scan int32 " << scan_config_name(scan_selected(OPTIGPU_INT32)) << "\n";
    f << "scan float " << scan_config_name(scan_selected(OPTIGPU_FLOAT32)) << "\n";
    f << "param transpose.group_rows " << transpose_group_rows() << "\n";
    return f ? OPTIGPU_OK : fail(OPTIGPU_ERR_INVALID_ARG, "tune_save: write failed");
}

optigpu_status optigpu_tune_load(const char *path)
{
    if (!path)
        return fail(OPTIGPU_ERR_INVALID_ARG, "tune_load: null path");
    std::ifstream f(path);
    if (!f)
        return fail(OPTIGPU_ERR_NOT_FOUND, std::string("tune_load: cannot open ") + path);
    std::string line;
    int applied = 0;
    while (std::getline(f, line)) {
        std::istringstream in(line);
        std::string kind;
        in >> kind;
        if (kind == "transpose") {
            int es = 0;
            in >> es;
            std::string name;
            std::getline(in >> std::ws, name);
            if (es != 2 && es != 4)
                continue;
            for (int c = 0; c < transpose_num_configs(size_t(es)); ++c)
                if (name == transpose_config_name(size_t(es), c)) {
                    transpose_select(size_t(es), c);
                    ++applied;
                }
        } else if (kind == "reduce") {
            std::string name;
            std::getline(in >> std::ws, name);
            for (int c = 0; c < reduce_num_configs(); ++c)
                if (name == reduce_config_name(c)) {
                    reduce_select(c);
                    ++applied;
                }
        } else if (kind == "batch") {
            std::string name;
            std::getline(in >> std::ws, name);
            for (int c = 0; c < batch_num_configs(); ++c)
                if (name == batch_config_name(c)) {
                    batch_select(c);
                    ++applied;
                }
        } else if (kind == "scan") {
            // "scan int32 <name>" or "scan float <name>"; a line without the
            // class names the form of both.
            std::string rest;
            std::getline(in >> std::ws, rest);
            int cls = -1;
            if (rest.rfind("int32 ", 0) == 0) {
                cls = OPTIGPU_INT32;
                rest = rest.substr(6);
            } else if (rest.rfind("float ", 0) == 0) {
                cls = OPTIGPU_FLOAT32;
                rest = rest.substr(6);
            }
            for (int c = 0; c < scan_num_configs(); ++c)
                if (rest == scan_config_name(c)) {
                    if (cls != OPTIGPU_FLOAT32)
                        scan_select(OPTIGPU_INT32, c);
                    if (cls != OPTIGPU_INT32)
                        scan_select(OPTIGPU_FLOAT32, c);
                    ++applied;
                }
        } else if (kind == "param") {
            std::string name;
            long long v = 0;
            in >> name >> v;
            if (optigpu_tune_set_param(name.c_str(), v) == OPTIGPU_OK)
                ++applied;
        }
    }
    return applied > 0 ? OPTIGPU_OK : fail(OPTIGPU_ERR_NOT_FOUND, "tune_load: no usable entries");
}

} // extern "C"
