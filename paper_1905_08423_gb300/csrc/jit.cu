// Plan-time specialisation of the class-program kernel.
//
// The interpreter in fastkern.cuh decodes each class's program (which product
// goes to which slot of the row of A P, and where each outer-product term
// lands in C) at run time.  For the classes that carry most of a plan's fine
// rows this file writes the same computation as straight-line CUDA -- slots
// become registers, the products become immediate offsets, and the outer
// product becomes a short loop over P(I,:) whose offsets come from a constant
// table -- compiles it for sm_103a
// with NVRTC together with fastkern.cuh, and loads it.  Other classes still
// run on the interpreter inside the same kernel.  Nothing here changes what is
// computed: the generated code performs the products of the program in the
// interpreter's order.
//
// NVRTC and the driver API are reached through dlopen and the runtime's
// driver entry points, so the library loads (and simply runs the interpreter)
// where either is missing.  Compiled modules are kept for the life of the
// process, keyed by device and source, and shared between plans; their cubins
// are also cached on disk (see cache_dir) so that a later process with the
// same classes skips the compile.
#include <cuda.h>
#include <dlfcn.h>
#include <sys/stat.h>
#include <unistd.h>
#include <nvrtc.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <chrono>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <string>
#include <vector>

#include "common.cuh"
#include "fastkern.cuh"
#include "fastkern_src.inc"  // kFastKernSource: the text of fastkern.cuh

namespace ptap {

size_t jit_smem_for(const ptap_plan* p);

namespace {

struct Nvrtc {
  bool ok = false;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&nvrtcVersion) version = nullptr;
};

struct Driver {
  bool ok = false;
  decltype(&cuModuleLoadData) load = nullptr;
  decltype(&cuModuleGetFunction) get_fn = nullptr;
  decltype(&cuFuncSetAttribute) set_attr = nullptr;
  decltype(&cuOccupancyMaxActiveBlocksPerMultiprocessor) occupancy = nullptr;
  decltype(&cuLaunchKernel) launch = nullptr;
};

std::mutex g_mu;
Nvrtc g_rtc;
Driver g_drv;
bool g_loaded = false;
std::map<std::pair<int, uint64_t>, CUfunction> g_cache;  // (device, source hash) -> function
std::map<void*, int> g_smem_attr;  // largest dynamic shared memory set on each function

template <class F>
bool sym(void* lib, const char* name, F& f) {
  f = (F)dlsym(lib, name);
  return f != nullptr;
}

template <class F>
bool drv(const char* name, F& f) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return false;
  }
  f = (F)p;
  return true;
}

void load_apis() {
  if (g_loaded) return;
  g_loaded = true;
  void* lib = nullptr;
  for (const char* n : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so"})
    if ((lib = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
  if (lib)
    g_rtc.ok = sym(lib, "nvrtcCreateProgram", g_rtc.create) && sym(lib, "nvrtcCompileProgram", g_rtc.compile) &&
               sym(lib, "nvrtcGetProgramLogSize", g_rtc.log_size) && sym(lib, "nvrtcGetProgramLog", g_rtc.log) &&
               sym(lib, "nvrtcGetCUBINSize", g_rtc.cubin_size) && sym(lib, "nvrtcGetCUBIN", g_rtc.cubin) &&
               sym(lib, "nvrtcDestroyProgram", g_rtc.destroy) && sym(lib, "nvrtcVersion", g_rtc.version);
  g_drv.ok = drv("cuModuleLoadData", g_drv.load) && drv("cuModuleGetFunction", g_drv.get_fn) &&
             drv("cuFuncSetAttribute", g_drv.set_attr) &&
             drv("cuOccupancyMaxActiveBlocksPerMultiprocessor", g_drv.occupancy) &&
             drv("cuLaunchKernel", g_drv.launch);
}

// Compiled modules also persist across processes, as cubin files named by
// the hash of everything that determines them: PTAP_JIT_CACHE names the
// directory (set but empty: no disk cache); by default $XDG_CACHE_HOME/ptap,
// else $HOME/.cache/ptap.  A file that fails to load is compiled again.
std::string cache_dir() {
  if (const char* d = getenv("PTAP_JIT_CACHE")) return d;
  if (const char* x = getenv("XDG_CACHE_HOME"); x && *x) return std::string(x) + "/ptap";
  if (const char* h = getenv("HOME"); h && *h) return std::string(h) + "/.cache/ptap";
  return "";
}

bool read_file(const std::string& path, std::vector<char>& out) {
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return false;
  std::vector<char> buf;
  char tmp[65536];
  size_t n;
  while ((n = fread(tmp, 1, sizeof tmp, f)) > 0) buf.insert(buf.end(), tmp, tmp + n);
  fclose(f);
  if (buf.empty()) return false;
  out.swap(buf);
  return true;
}

// mkdir -p, then write to a private temporary name and rename into place, so
// readers never see a partial file.  Failures only cost the next process a compile.
void write_file_atomic(const std::string& dir, const std::string& name, const std::vector<char>& data) {
  for (size_t i = 1; i <= dir.size(); ++i)
    if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
  const std::string path = dir + "/" + name;
  const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return;
  const bool ok = fwrite(data.data(), 1, data.size(), f) == data.size();
  if (fclose(f) != 0 || !ok || rename(tmp.c_str(), path.c_str()) != 0) remove(tmp.c_str());
}

uint64_t fnv64(const std::string& s) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (unsigned char c : s) h = (h ^ c) * 0x100000001b3ull;
  return h;
}

// printf-style append that never truncates.
void appendf(std::string& o, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  const int n = vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (n < 0) return;
  if (n < (int)sizeof buf) {
    o += buf;
    return;
  }
  std::string big((size_t)n + 1, '\0');
  va_start(ap, fmt);
  vsnprintf(&big[0], big.size(), fmt, ap);
  va_end(ap);
  big.resize((size_t)n);
  o += big;
}

// Code for one class program g (layout in fastkern.cuh).  The row of A P is
// straight-line code with its r slots in registers (Alg. 3); the outer
// product is a loop over the pI entries of P(I,:) whose body adds the r slots
// at offsets sigma(s, t) read from a per-class constant table (Alg. 8).  The
// loop keeps the code of a class near r accumulations instead of r * pI: the
// instruction cache, not the issue rate, limits how many classes pay off.
std::string gen_class(int cls, const uint8_t* g, int cached, int loc_bits) {
  const int na = g[0], r = g[1], pI = g[2];
  const uint8_t* pa = g + 8;
  const uint8_t* tsec = g + 8 + ((na + 7) & ~7);
  const uint8_t* ssec = tsec + 8 * na;
  std::string o;
  appendf(o, "static __constant__ unsigned char sg_%d[%d] = {", cls, pI * r);
  for (int s = 0; s < pI; ++s)
    for (int t = 0; t < r; ++t) appendf(o, "%d,", (int)ssec[t * 8 + s]);
  o += "};\n";
  appendf(o,
          "__device__ __forceinline__ void cls_%d(const FastArgs<V>& a, int32_t f, int32_t f1, int32_t i0,"
          " int32_t i1, V* acc, const int32_t* roff, int32_t I, const int32_t* rec) {\n",
          cls);
  o += "  const int lane = threadIdx.x & 31;\n  const bool valid = f + lane < f1;\n"
       "  const int32_t ra = a.A.rp[I];\n"
       "  const int32_t* Aci = a.A.ci + ra;\n  const V* Av = a.A.val + ra;\n  const V* Pv = a.P.val;\n"
       "  (void)rec;\n";
  if (cached == 1) o += "  const int32_t* Aq = a.aq + ra;\n  (void)Aci;\n";
  if (cached == 2) o += "  const int32_t* Rq = rec + lane;\n  (void)Aci;\n";
  for (int x = 0; x < na; ++x) {
    if (cached == 2)
      appendf(o, "  const V a%d = Av[%d];\n  const int32_t q%d = Rq[%d];\n", x, x, x, x * 32);
    else if (cached == 1)
      appendf(o, "  const V a%d = Av[%d];\n  const int32_t q%d = Aq[%d];\n", x, x, x, x);
    else
      appendf(o, "  const V a%d = Av[%d];\n  const int32_t q%d = a.P.rp[Aci[%d]];\n", x, x, x, x);
  }
  // slots of the row of A P, products summed in the interpreter's (a, b) order
  for (int t = 0; t < r; ++t) {
    appendf(o, "  V R%d = V(0);\n", t);
    for (int x = 0; x < na; ++x)
      for (int b = 0; b < pa[x]; ++b)
        if (tsec[x * 8 + b] == t) appendf(o, "  R%d += a%d * Pv[q%d + %d];\n", t, x, x, b);
  }
  // outer product: the next entry of P(I,:) is loaded while this one is added
  o += "  const int32_t rp = a.P.rp[I];\n";
  if (loc_bits > 0) {
    // compact chunks: i0 is the chunk number; row_loc packs (chunk, offset)
    o += "  int32_t ln = a.row_loc[a.P.ci[rp]];\n  V wn = a.P.val[rp];\n  (void)i1;\n  (void)roff;\n";
    appendf(o,
            "#pragma unroll 1\n  for (int s = 0; s < %d; ++s) {\n"
            "    const int32_t l = ln;\n    const V w = wn;\n"
            "    if (s + 1 < %d) {\n      ln = a.row_loc[a.P.ci[rp + s + 1]];\n      wn = a.P.val[rp + s + 1];\n"
            "    }\n"
            "    if (valid && (l >> %d) == i0) {\n      V* c = acc + (l & %d);\n"
            "      const unsigned char* sg = sg_%d + s * %d;\n",
            pI, pI, loc_bits, (1 << loc_bits) - 1, cls, r);
  } else if (cached == 2) {
    // the piece's record gives each lane's accumulator offsets (0xFFFF: none)
    appendf(o, "  const uint16_t* Ro = (const uint16_t*)(rec + %d) + lane;\n", na * 32);
    o += "  int32_t on = Ro[0];\n  V wn = a.P.val[rp];\n  (void)valid;\n  (void)i0;\n  (void)i1;\n"
         "  (void)roff;\n";
    appendf(o,
            "#pragma unroll 1\n  for (int s = 0; s < %d; ++s) {\n"
            "    const int32_t ofs = on;\n    const V w = wn;\n"
            "    if (s + 1 < %d) {\n      on = Ro[(s + 1) * 32];\n      wn = a.P.val[rp + s + 1];\n    }\n"
            "    if (ofs != 0xFFFF) {\n      V* c = acc + ofs;\n"
            "      const unsigned char* sg = sg_%d + s * %d;\n",
            pI, pI, cls, r);
  } else {
    o += "  int32_t in = a.P.ci[rp];\n  V wn = a.P.val[rp];\n";
    appendf(o,
            "#pragma unroll 1\n  for (int s = 0; s < %d; ++s) {\n"
            "    const int32_t i = in;\n    const V w = wn;\n"
            "    if (s + 1 < %d) {\n      in = a.P.ci[rp + s + 1];\n      wn = a.P.val[rp + s + 1];\n    }\n"
            "    if (valid && i >= i0 && i < i1) {\n      V* c = acc + roff[i - i0];\n"
            "      const unsigned char* sg = sg_%d + s * %d;\n",
            pI, pI, cls, r);
  }
  for (int t = 0; t < r; ++t) appendf(o, "      acc_fma(c + sg[%d], w, R%d);\n", t, t);
  o += "    }\n  }\n}\n";
  return o;
}


// Visits per class of one plan (from its pieces) and its class programs.
struct ClassTable {
  std::vector<int64_t> visits;
  std::vector<int32_t> off;
  std::vector<uint8_t> pool;
  int64_t total = 0;
  const uint8_t* prog(int k) const { return pool.data() + off[k]; }
  int len(int k) const {
    const uint8_t* g = prog(k);
    return 8 + ((g[0] + 7) & ~7) + 8 * g[0] + 8 * g[1];
  }
  std::string bytes(int k) const { return std::string((const char*)prog(k), (size_t)len(k)); }
};

int read_classes(ptap_plan* p, ClassTable& t) {
  cudaStream_t s = p->stream;
  std::vector<int32_t> meta(p->npieces);
  t.off.assign(p->nclasses, 0);
  PTAP_CUDA(cudaMemcpyAsync(meta.data(), p->piece_meta, meta.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaMemcpyAsync(t.off.data(), p->class_off, t.off.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  t.visits.assign(p->nclasses, 0);
  t.total = 0;
  int pool_len = 0;
  for (int32_t m : meta) {
    t.visits[m >> 6] += m & 63;
    t.total += m & 63;
  }
  for (int32_t o : t.off) pool_len = std::max(pool_len, o + p->class_maxlen);
  t.pool.assign(pool_len, 0);
  PTAP_CUDA(cudaMemcpy(t.pool.data(), p->class_pool, pool_len, cudaMemcpyDeviceToHost));
  return PTAP_OK;
}

// Source of a specialised kernel for the programs `hot` (in this order: the
// compiled-code numbers are positions in it).  kind 0: one product
// (ptap_jit_numeric); kind 1: a batch of products (ptap_jit_batch).
std::string build_source(int dtype, const std::vector<std::string>& hot, int cached, int loc_bits,
                         int block_threads, int kind) {
  std::string src = "#include \"fastkern.cuh\"\nusing namespace ptapk;\n";
  src += dtype == PTAP_F64 ? "typedef double V;\n" : "typedef float V;\n";
  for (size_t i = 0; i < hot.size(); ++i)
    src += gen_class((int)i, (const uint8_t*)hot[i].data(), cached, loc_bits);
  src += "struct Special {\n  __device__ bool operator()(const FastArgs<V>& a, int32_t slot, int32_t f, int32_t f1,"
         " int32_t i0, int32_t i1, V* acc, const int32_t* roff, int32_t I, const int32_t* rec) const {\n"
         "    switch (slot) {\n";
  for (size_t i = 0; i < hot.size(); ++i)
    appendf(src, "      case %d: cls_%d(a, f, f1, i0, i1, acc, roff, I, rec); return true;\n", (int)i, (int)i);
  src += "      default: return false;\n    }\n  }\n};\n";
  // FP32: 64 registers a thread, 1024 resident threads per SM.  FP64 code
  // holds twice the bytes in registers and spills at 64; 128 registers with
  // 512 resident threads measured faster.
  const int resident = dtype == PTAP_F64 ? 512 : 1024;
  const int minb = std::max(1, resident / block_threads);
  if (kind == 0) {
    appendf(src, "extern \"C\" __global__ void __launch_bounds__(%d, %d) ptap_jit_numeric(FastArgs<V> a) {\n",
            block_threads, minb);
    src += "  fast_kernel_body<V>(a, Special());\n}\n";
  } else {
    appendf(src,
            "extern \"C\" __global__ void __launch_bounds__(%d, %d) ptap_jit_batch(const FastArgs<V>* probs,"
            " const int32_t* items, int32_t nitems, int32_t* counter, int CH, int maxr, int max_rows,"
            " int prog_cap, V* rs) {\n",
            block_threads, minb);
    src += "  fast_batch_body<V>(probs, items, nitems, counter, CH, maxr, max_rows, prog_cap, rs, Special());\n}\n";
  }
  return src;
}

// Compiles `src` (or finds it in the process's or the disk cache) and returns
// the function `name` in *fn.  Caller holds g_mu.
int compile_or_load(const std::string& src, const char* name, CUfunction* fn_out) {
  int dev = 0;
  PTAP_CUDA(cudaGetDevice(&dev));
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo"};
  int rv_major = 0, rv_minor = 0;
  g_rtc.version(&rv_major, &rv_minor);
  std::string keytext = src + '\x01' + kFastKernSource + '\x01' + std::to_string(rv_major) + "." +
                        std::to_string(rv_minor);
  for (const char* o : opts) keytext += std::string("\x01") + o;
  const uint64_t key = fnv64(keytext);
  CUfunction fn = nullptr;
  auto it = g_cache.find({dev, key});
  const std::string dir = cache_dir();
  char fname[64];
  snprintf(fname, sizeof fname, "jit_%016llx_sm103a.cubin", (unsigned long long)key);
  // PTAP_JIT_SOURCE_DIR: also write the generated source there (jit_<key>.cu),
  // for reading and for offline compiles of the same code
  if (const char* sd = getenv("PTAP_JIT_SOURCE_DIR"); sd && *sd) {
    char sname[64];
    snprintf(sname, sizeof sname, "jit_%016llx.cu", (unsigned long long)key);
    write_file_atomic(sd, sname, std::vector<char>(src.begin(), src.end()));
  }
  std::vector<char> cached;
  if (it != g_cache.end()) {
    fn = it->second;
  } else if (!dir.empty() && read_file(dir + "/" + fname, cached)) {
    CUmodule mod = nullptr;
    if (g_drv.load(&mod, cached.data()) == CUDA_SUCCESS && g_drv.get_fn(&fn, mod, name) == CUDA_SUCCESS) {
      g_cache[{dev, key}] = fn;
    } else {
      fn = nullptr;
      cudaGetLastError();
    }
  }
  if (!fn) {
    nvrtcProgram prog;
    const char* hdr[1] = {kFastKernSource};
    const char* hname[1] = {"fastkern.cuh"};
    if (g_rtc.create(&prog, src.c_str(), "ptap_jit.cu", 1, hdr, hname) != NVRTC_SUCCESS) return PTAP_ERR_CUDA;
    const nvrtcResult rc = g_rtc.compile(prog, 3, opts);
    if (rc != NVRTC_SUCCESS) {
      if (getenv("PTAP_VERBOSE")) {
        size_t n = 0;
        g_rtc.log_size(prog, &n);
        std::string log(n, '\0');
        g_rtc.log(prog, &log[0]);
        fprintf(stderr, "ptap: NVRTC failed:\n%s\n", log.c_str());
      }
      g_rtc.destroy(&prog);
      return PTAP_ERR_CUDA;
    }
    size_t n = 0;
    g_rtc.cubin_size(prog, &n);
    std::vector<char> cubin(n);
    g_rtc.cubin(prog, cubin.data());
    g_rtc.destroy(&prog);
    CUmodule mod = nullptr;
    if (g_drv.load(&mod, cubin.data()) != CUDA_SUCCESS) return PTAP_ERR_CUDA;
    if (g_drv.get_fn(&fn, mod, name) != CUDA_SUCCESS) return PTAP_ERR_CUDA;
    g_cache[{dev, key}] = fn;
    if (!dir.empty()) write_file_atomic(dir, fname, cubin);
  }
  *fn_out = fn;
  return PTAP_OK;
}

// Raises the function's dynamic shared-memory limit to `smem` (a module is
// shared by plans: the attribute only grows) and returns its occupancy.
int set_smem_and_occupancy(CUfunction fn, int threads, size_t smem, int* per_sm) {
  int& attr = g_smem_attr[(void*)fn];
  if ((int)smem > attr) {
    if (g_drv.set_attr(fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)smem) != CUDA_SUCCESS)
      return PTAP_ERR_CUDA;
    attr = (int)smem;
  }
  *per_sm = 0;
  if (g_drv.occupancy(per_sm, fn, threads, smem) != CUDA_SUCCESS || *per_sm < 1) return PTAP_ERR_CUDA;
  return PTAP_OK;
}

}  // namespace

// Compiles `src` and publishes the kernel to the plan: its shared-memory
// limit and occupancy first, then jit_fn (release), which launches read.
// Runs on the caller's thread, or on p->jit_thread (background compile); it
// touches no library allocator.  On failure jit_fn stays null and the
// interpreter keeps serving the plan.
static void jit_compile_publish(ptap_plan* p, std::string src, int dev,
                                std::chrono::steady_clock::time_point t0) {
  CUfunction fn = nullptr;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    if (compile_or_load(src, "ptap_jit_numeric", &fn) != PTAP_OK) return;
    // The compiled classes keep their rows of A P in registers, so the
    // interpreted ones use a global scratch instead of shared memory: the
    // accumulator alone sets the shared-memory footprint.
    if (set_smem_and_occupancy(fn, p->cfg.block_threads, p->jit_smem, &per_sm) != PTAP_OK) return;
  }
  p->jit_per_sm = std::min(per_sm, p->jit_per_sm);  // jit_per_sm holds the bound the scratch was sized for
  p->jit_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  p->jit_fn.store((void*)fn, std::memory_order_release);
}

// Picks the classes with the most visited rows and generates the specialised
// kernel, then compiles and loads it -- at once, or, with specialize_async, in
// a background thread while numeric calls run the interpreter.  Returns
// PTAP_OK, or any error (the caller then keeps the interpreter).
int jit_prepare(ptap_plan* p) {
  {
    std::lock_guard<std::mutex> lock(g_mu);
    load_apis();
  }
  if (!g_rtc.ok || !g_drv.ok || !p->fast || p->nclasses <= 0) return PTAP_ERR_UNSUPPORTED;
  cudaStream_t s = p->stream;
  const auto t0 = std::chrono::steady_clock::now();
  ClassTable t;
  PTAP_TRY(read_classes(p, t));
  // Class ids come from a concurrent deduplication and differ between runs;
  // the generated source must not, or the disk cache would never hit.  So
  // classes are ranked by visits with ties broken by program bytes, and the
  // compiled ones are numbered in program-byte order; a device table maps a
  // plan's class ids to those numbers.
  std::vector<int> order(p->nclasses);
  for (int k = 0; k < p->nclasses; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    return t.visits[x] != t.visits[y] ? t.visits[x] > t.visits[y] : t.bytes(x) < t.bytes(y);
  });
  std::vector<int> hot;
  int64_t covered = 0;
  for (int k : order) {
    if ((int)hot.size() >= p->cfg.jit_max_classes || covered >= t.total * 99 / 100 || t.visits[k] == 0) break;
    hot.push_back(k);
    covered += t.visits[k];
  }
  if (hot.empty()) return PTAP_ERR_UNSUPPORTED;
  std::sort(hot.begin(), hot.end(), [&](int x, int y) { return t.bytes(x) < t.bytes(y); });
  std::vector<std::string> progs;
  for (int k : hot) progs.push_back(t.bytes(k));
  std::string src = build_source(p->dtype, progs, p->index_mode(), p->compact ? p->loc_bits : 0,
                                 p->cfg.block_threads, 0);
  // Resources the launch needs, sized before the compile (on this thread:
  // the allocator is not shared with the background thread).  The scratch
  // takes the resident-CTA bound that the thread count allows.
  p->jit_smem = jit_smem_for(p);
  const int bound_per_sm = std::max(1, 2048 / p->cfg.block_threads);
  p->jit_per_sm = bound_per_sm;
  const size_t vb = p->dtype == PTAP_F64 ? 8 : 4;
  const int64_t ctas = std::min<int64_t>(p->nchunks, (int64_t)num_sms() * bound_per_sm);
  void* rs = nullptr;
  PTAP_TRY(p->mem.get(&rs, (size_t)std::max<int64_t>(ctas, 1) * p->cfg.block_threads *
                               std::max(p->class_maxr, 1) * vb));
  std::vector<int32_t> slot(p->nclasses, -1);
  for (size_t i = 0; i < hot.size(); ++i) slot[hot[i]] = (int32_t)i;
  int32_t* dslot = nullptr;
  PTAP_TRY(p->mem.get_n(&dslot, p->nclasses));
  PTAP_CUDA(cudaMemcpyAsync(dslot, slot.data(), slot.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  p->jit_slot = dslot;
  p->jit_rs = rs;
  p->jit_classes = (int)hot.size();
  p->jit_coverage = t.total ? (double)covered / (double)t.total : 0.0;
  int dev = 0;
  PTAP_CUDA(cudaGetDevice(&dev));
  if (p->cfg.jit_async) {
    p->jit_thread = new (std::nothrow) std::thread(jit_compile_publish, p, std::move(src), dev, t0);
    if (!p->jit_thread) jit_compile_publish(p, std::move(src), dev, t0);
    return PTAP_OK;
  }
  jit_compile_publish(p, std::move(src), dev, t0);
  return p->jit_fn.load(std::memory_order_acquire) ? PTAP_OK : PTAP_ERR_CUDA;
}

int jit_launch(ptap_plan* p, void* fn, const void* args, int grid, cudaStream_t s) {
  void* params[1] = {const_cast<void*>(args)};
  if (g_drv.launch((CUfunction)fn, grid, 1, 1, p->cfg.block_threads, 1, 1, (unsigned)p->jit_smem, (CUstream)s,
                   params, nullptr) != CUDA_SUCCESS)
    return PTAP_ERR_CUDA;
  return PTAP_OK;
}

// Specialisation for a batch: the class programs of all `count` plans are
// pooled by their bytes (identical structure classes of different products
// share one compiled body), visits are summed over the plans, and the most
// visited `max_classes` programs are compiled into ptap_jit_batch.  For each
// plan, slots[q] receives a device table (from `mem`) mapping its class ids
// to compiled numbers or -1.  All plans must agree on the cached indices; compact
// chunks are not specialised.
int jit_prepare_batch(ptap_plan* const* plans, int count, int max_classes, int threads, Tracker& mem,
                      cudaStream_t s, void** fn_out, std::vector<int32_t*>& slots, int* nhot,
                      double* coverage) {
  std::lock_guard<std::mutex> lock(g_mu);
  load_apis();
  if (!g_rtc.ok || !g_drv.ok || count <= 0) return PTAP_ERR_UNSUPPORTED;
  const int cached = plans[0]->index_mode();
  std::vector<ClassTable> tabs(count);
  std::map<std::string, int64_t> pooled;
  int64_t total = 0;
  for (int q = 0; q < count; ++q) {
    ptap_plan* p = plans[q];
    if (!p->fast || p->compact || p->index_mode() != cached || p->nclasses <= 0) return PTAP_ERR_UNSUPPORTED;
    PTAP_TRY(read_classes(p, tabs[q]));
    for (int k = 0; k < p->nclasses; ++k) pooled[tabs[q].bytes(k)] += tabs[q].visits[k];
    total += tabs[q].total;
  }
  std::vector<std::pair<int64_t, std::string>> ranked;
  for (auto& kv : pooled) ranked.push_back({kv.second, kv.first});
  std::sort(ranked.begin(), ranked.end(), [](const auto& x, const auto& y) {
    return x.first != y.first ? x.first > y.first : x.second < y.second;
  });
  std::vector<std::string> hot;
  int64_t covered = 0;
  for (auto& r : ranked) {
    if ((int)hot.size() >= max_classes || covered >= total * 99 / 100 || r.first == 0) break;
    hot.push_back(r.second);
    covered += r.first;
  }
  if (hot.empty()) return PTAP_ERR_UNSUPPORTED;
  std::sort(hot.begin(), hot.end());
  std::map<std::string, int32_t> number;
  for (size_t i = 0; i < hot.size(); ++i) number[hot[i]] = (int32_t)i;
  const std::string src = build_source(plans[0]->dtype, hot, cached, 0, threads, 1);
  CUfunction fn = nullptr;
  PTAP_TRY(compile_or_load(src, "ptap_jit_batch", &fn));
  slots.assign(count, nullptr);
  for (int q = 0; q < count; ++q) {
    std::vector<int32_t> slot(plans[q]->nclasses, -1);
    for (int k = 0; k < plans[q]->nclasses; ++k) {
      auto it = number.find(tabs[q].bytes(k));
      if (it != number.end()) slot[k] = it->second;
    }
    PTAP_TRY(mem.get_n(&slots[q], (int64_t)slot.size()));
    PTAP_CUDA(cudaMemcpyAsync(slots[q], slot.data(), slot.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  }
  PTAP_CUDA(cudaStreamSynchronize(s));
  *fn_out = (void*)fn;
  *nhot = (int)hot.size();
  *coverage = total ? (double)covered / (double)total : 0.0;
  return PTAP_OK;
}

int jit_occupancy(void* fn, int threads, size_t smem, int* per_sm) {
  std::lock_guard<std::mutex> lock(g_mu);
  return set_smem_and_occupancy((CUfunction)fn, threads, smem, per_sm);
}

int jit_launch_raw(void* fn, void** params, int grid, int threads, size_t smem, cudaStream_t s) {
  if (g_drv.launch((CUfunction)fn, grid, 1, 1, threads, 1, 1, (unsigned)smem, (CUstream)s, params, nullptr) !=
      CUDA_SUCCESS)
    return PTAP_ERR_CUDA;
  return PTAP_OK;
}

}  // namespace ptap
