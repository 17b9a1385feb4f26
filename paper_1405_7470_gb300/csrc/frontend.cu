// General front end for elementwise instructions: a loop domain of one or two inames and
// one assignment whose right-hand side is an arithmetic expression (Section 2.1), turned
// into a CUDA kernel at run time, as the paper's code generator does:
//
//   split_iname (Eq. 1)    the domain is cut into tiles; for every tile the kernel
//                          dispatches between bulk code without any guard and separate
//                          edge code (a tile cut by one bound) and corner code (cut by
//                          both bounds of a 2-D domain), each with only the guards it
//                          needs (the extra argument of split_iname in Section 2.4);
//   vec / ilp / unr        bulk code moves 16-byte vectors along the innermost iname,
//                          `unroll` vectors per thread and tile, loads first;
//   data layout            arrays are dense row-major over the inames they are indexed by
//                          (a 1-D array inside a 2-D domain is broadcast along the other).
//
// Every operation is one IEEE single-precision operation rounded to nearest (the
// generated code calls __fadd_rn and friends and is compiled without contraction), so the
// result equals the plain loop over the domain bit for bit, whatever the tiling.
//
// Code generation uses NVRTC (loaded on first use), the module is loaded with the runtime's
// library API; compiled kernels are cached per generated source for the process's life.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "lc_internal.h"

namespace lc {

// ------------------------------------------------------------------ NVRTC, loaded on demand

struct Nvrtc {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    bool ok = false;
};

static const Nvrtc &nvrtc()
{
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr)
                break;
        if (!h)
            return;
        n.create = (decltype(n.create))dlsym(h, "nvrtcCreateProgram");
        n.compile = (decltype(n.compile))dlsym(h, "nvrtcCompileProgram");
        n.log_size = (decltype(n.log_size))dlsym(h, "nvrtcGetProgramLogSize");
        n.log = (decltype(n.log))dlsym(h, "nvrtcGetProgramLog");
        n.cubin_size = (decltype(n.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
        n.cubin = (decltype(n.cubin))dlsym(h, "nvrtcGetCUBIN");
        n.destroy = (decltype(n.destroy))dlsym(h, "nvrtcDestroyProgram");
        n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
    });
    return n;
}

// ------------------------------------------------------------------ code generation

static std::string fbits(double v)
{
    float f = (float)v;  // the constant as a binary32 value (nearest-even from its double)
    uint32_t b;
    memcpy(&b, &f, 4);
    char s[40];
    snprintf(s, sizeof s, "__uint_as_float(0x%08xu)", b);
    return s;
}

// The expression for one element; leaf(k) gives the C expression of array k's value.
template <typename Leaf>
static std::string expr(const Elementwise &P, int n, const Leaf &leaf)
{
    const EwNode &x = P.nodes[n];
    switch (x.op) {
    case EW_LOAD: return leaf(x.arg);
    case EW_PARAM: return "p" + std::to_string(x.arg);
    case EW_CONST: return fbits(x.val);
    case EW_NEG: return "(-" + expr(P, x.a, leaf) + ")";
    case EW_ADD: return "__fadd_rn(" + expr(P, x.a, leaf) + ", " + expr(P, x.b, leaf) + ")";
    case EW_SUB: return "__fsub_rn(" + expr(P, x.a, leaf) + ", " + expr(P, x.b, leaf) + ")";
    case EW_MUL: return "__fmul_rn(" + expr(P, x.a, leaf) + ", " + expr(P, x.b, leaf) + ")";
    default: return "__fdiv_rn(" + expr(P, x.a, leaf) + ", " + expr(P, x.b, leaf) + ")";
    }
}

static constexpr int kEwThreads = 256;

// CUDA source of the kernel for a program, unroll factor and edge handling.
static std::string generate(const Elementwise &P, int ndim, int unroll, bool edge_code)
{
    const int na = (int)P.arrays.size();
    std::string s;
    s += "// generated by the lc elementwise front end\n";
    s += "extern \"C\" __global__ void __launch_bounds__(256) lc_elementwise(float *__restrict__ a0";
    for (int k = 1; k < na; ++k)
        s += ", const float *__restrict__ a" + std::to_string(k);
    for (size_t k = 0; k < P.params.size(); ++k)
        s += ", float p" + std::to_string(k);
    s += ", long long n0, long long n1, int vec)\n{\n";
    const std::string U = std::to_string(unroll);
    if (ndim == 1) {
        // tiles of T = 256 * 4 * U elements: bulk code (vectors, no guard) or edge code
        s += "    const long long T = 1024LL * " + U + ";\n";
        s += "    const long long ntiles = (n0 + T - 1) / T;\n";
        s += "    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {\n";
        s += "        const long long base = t * T;\n";
        s += "        if (vec && base + T <= n0) {\n";
        for (int k = 1; k < na; ++k)
            s += "            float4 x" + std::to_string(k) + "[" + U + "];\n";
        s += "#pragma unroll\n            for (int u = 0; u < " + U + "; ++u) {\n";
        s += "                const long long q = base / 4 + threadIdx.x + 256 * u;\n";
        for (int k = 1; k < na; ++k)
            s += "                x" + std::to_string(k) + "[u] = __ldcs(reinterpret_cast<const float4 *>(a" +
                 std::to_string(k) + ") + q);\n";
        s += "            }\n";
        s += "#pragma unroll\n            for (int u = 0; u < " + U + "; ++u) {\n";
        s += "                float4 r;\n";
        for (const char *c : {"x", "y", "z", "w"}) {
            std::string comp = c;
            s += "                r." + comp + " = " +
                 expr(P, P.root, [&](int k) { return "x" + std::to_string(k) + "[u]." + comp; }) + ";\n";
        }
        s += "                __stcs(reinterpret_cast<float4 *>(a0) + base / 4 + threadIdx.x + 256 * u, r);\n";
        s += "            }\n";
        s += "        } else {\n";
        if (edge_code) {
            s += "            for (long long i = base + threadIdx.x; i < n0 && i < base + T; i += 256)\n";
            s += "                a0[i] = " + expr(P, P.root, [&](int k) { return "a" + std::to_string(k) + "[i]"; }) + ";\n";
        } else {
            // tail-free variant (assumption: n0 is a multiple of the tile): unguarded scalar code
            s += "            for (long long i = base + threadIdx.x; i < base + T; i += 256)\n";
            s += "                a0[i] = " + expr(P, P.root, [&](int k) { return "a" + std::to_string(k) + "[i]"; }) + ";\n";
        }
        s += "        }\n    }\n}\n";
        return s;
    }
    // 2-D: tiles of TI = 4 * U rows x TJ = 256 columns; thread (ty, tx) = (tid / 64, tid % 64)
    // covers rows ty + 4u and columns 4 tx .. 4 tx + 3 of the tile
    auto idx = [&](int k, const std::string &i, const std::string &j) -> std::string {
        const std::vector<int> &d = P.arrays[k].dims;
        if (d.size() == 2)
            return i + " * n1 + " + j;
        return d[0] == 0 ? i : j;
    };
    s += "    const int TI = 4 * " + U + ", TJ = 256;\n";
    s += "    const long long mi = (n0 + TI - 1) / TI, mj = (n1 + TJ - 1) / TJ;\n";
    s += "    const int ty = threadIdx.x >> 6, tx = threadIdx.x & 63;\n";
    s += "    for (long long t = blockIdx.x; t < mi * mj; t += gridDim.x) {\n";
    s += "        const long long ti = t / mj, tj = t - ti * mj;\n";
    s += "        const long long i0 = ti * TI + ty, j0 = tj * TJ + 4 * tx;\n";
    s += "        const bool full_i = (ti + 1) * TI <= n0, full_j = (tj + 1) * TJ <= n1;\n";
    // vector code: bulk (no guard) and the edge cut along i (row guard only)
    auto vector_body = [&](bool guard_i) {
        std::string b;
        b += "#pragma unroll\n            for (int u = 0; u < " + U + "; ++u) {\n";
        b += "                const long long i = i0 + 4 * u;\n";
        if (guard_i)
            b += "                if (i >= n0) break;\n";
        for (int k = 1; k < na; ++k) {
            const std::vector<int> &d = P.arrays[k].dims;
            const std::string nm = "x" + std::to_string(k);
            if (d.size() == 1 && d[0] == 0)
                b += "                const float " + nm + "s = a" + std::to_string(k) + "[i];\n";
            else
                b += "                const float4 " + nm + " = __ldcs(reinterpret_cast<const float4 *>(a" +
                     std::to_string(k) + " + " + idx(k, "i", "j0") + "));\n";
        }
        b += "                float4 r;\n";
        for (const char *c : {"x", "y", "z", "w"}) {
            std::string comp = c;
            b += "                r." + comp + " = " + expr(P, P.root, [&](int k) {
                     const std::vector<int> &d = P.arrays[k].dims;
                     return (d.size() == 1 && d[0] == 0) ? "x" + std::to_string(k) + "s"
                                                         : "x" + std::to_string(k) + "." + comp;
                 }) + ";\n";
        }
        b += "                __stcs(reinterpret_cast<float4 *>(a0 + i * n1 + j0), r);\n";
        b += "            }\n";
        return b;
    };
    // scalar code with the guards of an edge or corner tile
    auto scalar_body = [&](bool guard_i, bool guard_j) {
        std::string b;
        b += "#pragma unroll\n            for (int u = 0; u < " + U + "; ++u) {\n";
        b += "                const long long i = i0 + 4 * u;\n";
        if (guard_i)
            b += "                if (i >= n0) break;\n";
        b += "                for (int c = 0; c < 4; ++c) {\n";
        b += "                    const long long j = j0 + c;\n";
        if (guard_j)
            b += "                    if (j >= n1) break;\n";
        b += "                    a0[i * n1 + j] = " +
             expr(P, P.root, [&](int k) { return "a" + std::to_string(k) + "[" + idx(k, "i", "j") + "]"; }) + ";\n";
        b += "                }\n            }\n";
        return b;
    };
    s += "        if (vec && full_i && full_j) {          // bulk: no guard\n" + vector_body(false);
    s += "        } else if (vec && full_j) {             // edge cut by n0: row guard\n" + vector_body(true);
    s += "        } else if (full_i) {                    // edge cut by n1: column guard\n" + scalar_body(false, true);
    s += "        } else {                                // corner: both guards\n" + scalar_body(true, true);
    s += "        }\n    }\n}\n";
    return s;
}

// ------------------------------------------------------------------ compiled kernel cache

struct EwModule {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t fn = nullptr;
};

static std::mutex g_ew_mu;
static std::map<std::pair<int, std::string>, std::shared_ptr<EwModule>> g_ew_cache;  // (device, source)

static lc_status compile_ew(const std::string &src, cudaKernel_t *fn)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e);
    std::lock_guard<std::mutex> lk(g_ew_mu);
    auto key = std::make_pair(dev, src);
    auto it = g_ew_cache.find(key);
    if (it != g_ew_cache.end()) {
        *fn = it->second->fn;
        return LC_OK;
    }
    const Nvrtc &nv = nvrtc();
    if (!nv.ok)
        return LC_ERR_UNSUPPORTED;  // no run-time compiler on this machine
    nvrtcProgram prog;
    if (nv.create(&prog, src.c_str(), "lc_elementwise.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return LC_ERR_UNSUPPORTED;
    const char *opts[] = {"--gpu-architecture=sm_103a", "--fmad=false", "-std=c++17", "-default-device"};
    nvrtcResult rc = nv.compile(prog, 4, opts);
    std::vector<char> cubin;
    if (rc == NVRTC_SUCCESS) {
        size_t n = 0;
        if (nv.cubin_size(prog, &n) == NVRTC_SUCCESS && n > 0) {
            cubin.resize(n);
            if (nv.cubin(prog, cubin.data()) != NVRTC_SUCCESS)
                cubin.clear();
        }
    }
    nv.destroy(&prog);
    if (cubin.empty())
        return LC_ERR_UNSUPPORTED;
    auto m = std::make_shared<EwModule>();
    e = cudaLibraryLoadData(&m->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess)
        e = cudaLibraryGetKernel(&m->fn, m->lib, "lc_elementwise");
    if (e != cudaSuccess)
        return cuda_fail(e);
    g_ew_cache[key] = m;
    *fn = m->fn;
    return LC_OK;
}

struct EwPlan {
    int unroll, ndim;
    bool vec, edge_code;
    long long ntiles;
    int grid;
};

// Validate a descriptor for an elementwise kernel and sizes; no launch.
static lc_status ew_plan(const Kernel &K, const lc_variant *v, const int64_t *ext, EwPlan &p, bool need_device)
{
    if (!v || v->struct_size != sizeof(lc_variant) || !ext)
        return LC_ERR_INVALID_ARGUMENT;
    const Elementwise &P = K.ew;
    p.ndim = (int)K.inames.size();
    for (int d = 0; d < p.ndim; ++d)
        if (ext[d] < 0)
            return LC_ERR_INVALID_ARGUMENT;
    if (v->engine != LC_ENGINE_SIMT || v->precision != LC_PREC_FP32 || v->layout != LC_LAYOUT_ELEM_MAJOR ||
        !(v->unroll == 1 || v->unroll == 2 || v->unroll == 4 || v->unroll == 8) ||
        !(v->elems_per_thread == 1 || v->elems_per_thread == 4) || v->prefetch_smem != 0 || v->stages != 1 ||
        v->split_i != 0 || v->ctas_per_sm < 0 || v->ctas_per_sm > 32 || v->max_ctas < 0 || v->out_buffers != 0 ||
        v->store_rows != 0 || v->mma_order != 0 || v->a_operand != 0 || (v->tail_free != 0 && v->tail_free != 1))
        return LC_ERR_INVALID_VARIANT;
    p.unroll = v->unroll;
    const long long tile = p.ndim == 1 ? 1024LL * p.unroll : 256;  // along the innermost iname
    if (v->tile_e != 0 && v->tile_e != tile)
        return LC_ERR_INVALID_VARIANT;
    p.edge_code = true;
    if (v->tail_free) {
        // guard-free code only for a 1-D domain whose bound is assumed a multiple of the tile
        bool implied = false;
        for (const auto &a : K.assumptions)
            if (p.ndim == 1 && a.param == K.bounds[0] && a.op == 0 && a.k % tile == 0)
                implied = true;
        if (!implied)
            return LC_ERR_INVALID_VARIANT;
        p.edge_code = false;
    }
    for (const auto &a : K.assumptions) {
        long long val = -1;
        for (int d = 0; d < p.ndim; ++d)
            if (K.bounds[d] == a.param)
                val = ext[d];
        bool ok = true;
        switch (a.op) {
        case 0: ok = val % a.k == 0; break;
        case 1: ok = val >= a.k; break;
        case 2: ok = val > a.k; break;
        case 3: ok = val <= a.k; break;
        case 4: ok = val < a.k; break;
        case 5: ok = val == a.k; break;
        }
        if (!ok)
            return LC_ERR_ASSUMPTION;
    }
    const long long n0 = ext[0], n1 = p.ndim == 2 ? ext[1] : 1;
    p.vec = v->elems_per_thread == 4 && (p.ndim == 1 || n1 % 4 == 0);
    p.ntiles = p.ndim == 1 ? (n0 + tile - 1) / tile : ((n0 + 4LL * p.unroll - 1) / (4LL * p.unroll)) * ((n1 + 255) / 256);
    const int sms = need_device ? sm_count() : 148;
    if (need_device && sms <= 0)
        return LC_ERR_NO_DEVICE;
    long long grid = std::max<long long>(1, std::min<long long>(p.ntiles, (long long)(v->ctas_per_sm ? v->ctas_per_sm : 4) * sms));
    if (v->max_ctas > 0)
        grid = std::min<long long>(grid, v->max_ctas);
    p.grid = (int)grid;
    (void)P;
    return LC_OK;
}

lc_status ew_validate(const Kernel &K, const lc_variant *v, const int64_t *extents, bool need_device, int *grid,
                      long long *ntiles)
{
    if (K.kind != KIND_ELEMENTWISE)
        return LC_ERR_UNSUPPORTED;
    EwPlan p;
    lc_status st = ew_plan(K, v, extents, p, need_device);
    if (st == LC_OK) {
        *grid = p.grid;
        *ntiles = p.ntiles;
    }
    return st;
}

}  // namespace lc

using namespace lc;

extern "C" {

lc_status lc_kernel_signature(const lc_kernel *kh, int32_t *n_arrays, int32_t *n_params, int32_t *n_dims)
{
    if (!kh || !n_arrays || !n_params || !n_dims)
        return LC_ERR_INVALID_ARGUMENT;
    const Kernel &K = kh->k;
    if (K.kind == KIND_ELEMENTWISE) {
        *n_arrays = (int32_t)K.ew.arrays.size();
        *n_params = (int32_t)K.ew.params.size();
    } else {
        *n_arrays = K.kind == KIND_GEO ? 4 : K.kind == KIND_LIFT ? 6 : 3;
        *n_params = 0;
    }
    *n_dims = (int32_t)K.inames.size();
    return LC_OK;
}

lc_status lc_kernel_arg_name(const lc_kernel *kh, int32_t what, int32_t index, char *buf, size_t cap)
{
    if (!kh || !buf || cap == 0 || index < 0)
        return LC_ERR_INVALID_ARGUMENT;
    const Kernel &K = kh->k;
    std::string name;
    if (what == 2) {
        if (index >= (int)K.inames.size())
            return LC_ERR_INVALID_ARGUMENT;
        name = K.bounds[index];
    } else if (K.kind == KIND_ELEMENTWISE) {
        if (what == 0 && index < (int)K.ew.arrays.size())
            name = K.ew.arrays[index].name;
        else if (what == 1 && index < (int)K.ew.params.size())
            name = K.ew.params[index];
        else
            return LC_ERR_INVALID_ARGUMENT;
    } else {
        std::vector<std::string> arrs = {K.out_name, K.d_name, K.u_name};
        if (K.kind == KIND_GEO)
            arrs.push_back(K.g_name);
        if (K.kind == KIND_LIFT)
            arrs = {K.out_name, K.d_name, K.fmask_name, K.vmap_name, K.s_name, K.u_name};
        if (what != 0 || index >= (int)arrs.size())
            return LC_ERR_INVALID_ARGUMENT;
        name = arrs[index];
    }
    const size_t n = std::min(cap - 1, name.size());
    memcpy(buf, name.data(), n);
    buf[n] = 0;
    return n < name.size() ? LC_ERR_BUFFER_TOO_SMALL : LC_OK;
}

lc_status lc_elementwise_source(const lc_kernel *kh, const lc_variant *v, const int64_t *extents, char *buf,
                                size_t cap, size_t *needed)
{
    if (!kh)
        return LC_ERR_INVALID_ARGUMENT;
    if (kh->k.kind != KIND_ELEMENTWISE)
        return LC_ERR_UNSUPPORTED;
    EwPlan p;
    lc_status st = ew_plan(kh->k, v, extents, p, false);
    if (st != LC_OK)
        return st;
    const std::string src = generate(kh->k.ew, p.ndim, p.unroll, p.edge_code);
    if (needed)
        *needed = src.size() + 1;
    if (!buf || cap == 0)
        return LC_ERR_BUFFER_TOO_SMALL;
    const size_t n = std::min(cap - 1, src.size());
    memcpy(buf, src.data(), n);
    buf[n] = 0;
    return n < src.size() ? LC_ERR_BUFFER_TOO_SMALL : LC_OK;
}

lc_status lc_elementwise(const lc_kernel *kh, const lc_variant *v, const int64_t *extents, void *const *arrays,
                         const double *params, void *stream)
{
    if (!kh || !v || !extents || !arrays)
        return LC_ERR_INVALID_ARGUMENT;
    const Kernel &K = kh->k;
    if (K.kind != KIND_ELEMENTWISE)
        return LC_ERR_UNSUPPORTED;
    const Elementwise &P = K.ew;
    if (!P.params.empty() && !params)
        return LC_ERR_INVALID_ARGUMENT;
    EwPlan p;
    lc_status st = ew_plan(K, v, extents, p, true);
    if (st != LC_OK)
        return st;
    const long long n0 = extents[0], n1 = p.ndim == 2 ? extents[1] : 1;
    const long long total = n0 * n1;
    // array sizes: the product of the extents of the inames each is indexed by
    std::vector<long long> bytes(P.arrays.size());
    for (size_t k = 0; k < P.arrays.size(); ++k) {
        long long cnt = 1;
        for (int d : P.arrays[k].dims)
            cnt *= extents[d];
        bytes[k] = cnt * 4;
        if (cnt > 0 && !arrays[k])
            return LC_ERR_INVALID_ARGUMENT;
        const uintptr_t a = (uintptr_t)arrays[k];
        if ((a & 3u) || (p.vec && (a & 15u)))
            return LC_ERR_MISALIGNED;
    }
    // the output must not overlap an input
    for (size_t k = 1; k < P.arrays.size(); ++k) {
        const uintptr_t o0 = (uintptr_t)arrays[0], o1 = o0 + bytes[0];
        const uintptr_t x0 = (uintptr_t)arrays[k], x1 = x0 + bytes[k];
        if (bytes[0] > 0 && bytes[k] > 0 && o0 < x1 && x0 < o1)
            return LC_ERR_INVALID_ARGUMENT;
    }
    int major = 0, minor = 0;
    if (current_cc(&major, &minor) != 0 || major != 10 || minor != 3)
        return LC_ERR_NO_DEVICE;
    if (total == 0)
        return LC_OK;
    cudaKernel_t fn = nullptr;
    st = compile_ew(generate(P, p.ndim, p.unroll, p.edge_code), &fn);
    if (st != LC_OK)
        return st;
    std::vector<void *> args;
    std::vector<float> pf(P.params.size());
    for (size_t k = 0; k < P.params.size(); ++k)
        pf[k] = (float)params[k];  // binary32 nearest to the given value
    for (size_t k = 0; k < P.arrays.size(); ++k)
        args.push_back(const_cast<void **>(&arrays[k]));
    for (size_t k = 0; k < pf.size(); ++k)
        args.push_back(&pf[k]);
    long long a_n0 = n0, a_n1 = n1;
    int vec = p.vec ? 1 : 0;
    args.push_back(&a_n0);
    args.push_back(&a_n1);
    args.push_back(&vec);
    cudaError_t e = cudaLaunchKernel((const void *)fn, dim3(p.grid), dim3(kEwThreads), args.data(), 0,
                                     (cudaStream_t)stream);
    return e == cudaSuccess ? LC_OK : cuda_fail(e);
}

}  // extern "C"
