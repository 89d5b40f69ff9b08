// Run-time specialisation of the BSSN stage kernel (Sec. 3.2.3: besides the
// code generator, the run-time library compiles loop kernels once the
// parameter values are known, to cut code and register overhead).
//
// chemora_system_specialize writes, for one system, a small CUDA source that
// instantiates the device body of its launch shape (bssn_kernels.cuh) with
//   * the grid extents, ghost width and strides as literals (every neighbour
//     offset becomes an immediate, no stride arithmetic in registers),
//   * the scalars 1/(12h), 1/(12h^2), 1/(144h^2), the dissipation scale and
//     the gauge parameters as compile-time constants (exact hexadecimal
//     literals, so the arithmetic is the ahead-of-time kernel's), and
//   * one kernel per Runge-Kutta stage mode (the update's branches fold),
//     while the numeric constants of the bodies stay a kernel parameter
//     (KTable) so that adds and multiplies keep their fma form,
// compiles it with NVRTC for the device's architecture, loads the cubins as
// CUDA libraries and launches them in place of the ahead-of-time kernels.
// NVRTC is loaded with dlopen on first use, so the library itself does not
// depend on it.  Compiled cubins are cached on disk under a hash of the
// source, the embedded headers, the options and the NVRTC version.
#include <dlfcn.h>
#include <nvrtc.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <chrono>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace chemora {

namespace {

struct JitHeader {
  const char* name;
  const char* const* chunks;
  int nchunks;
};
#include "generated/jit_sources.inc"  // kJitHeaders[], kNumJitHeaders

constexpr int kModes = 5;

struct Nvrtc {
  bool ok = false;
  std::string why;
  decltype(&nvrtcVersion) version = nullptr;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&nvrtcGetErrorString) error_string = nullptr;
  int major = 0, minor = 0;
};

template <class F>
static bool sym(void* h, const char* name, F* out) {
  *out = reinterpret_cast<F>(dlsym(h, name));
  return *out != nullptr;
}

const Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    std::vector<std::string> cands = {"libnvrtc.so.13", "libnvrtc.so"};
    for (const char* env : {"CUDA_HOME", "CUDA_PATH"}) {
      const char* p = getenv(env);
      if (p && *p) cands.push_back(std::string(p) + "/lib64/libnvrtc.so.13");
    }
    cands.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
    void* h = nullptr;
    for (const std::string& c : cands)
      if ((h = dlopen(c.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) {
      n.why = "NVRTC (libnvrtc.so.13) not found";
      return;
    }
    bool ok = sym(h, "nvrtcVersion", &n.version) && sym(h, "nvrtcCreateProgram", &n.create) &&
              sym(h, "nvrtcCompileProgram", &n.compile) &&
              sym(h, "nvrtcGetProgramLogSize", &n.log_size) && sym(h, "nvrtcGetProgramLog", &n.log) &&
              sym(h, "nvrtcGetCUBINSize", &n.cubin_size) && sym(h, "nvrtcGetCUBIN", &n.cubin) &&
              sym(h, "nvrtcDestroyProgram", &n.destroy) &&
              sym(h, "nvrtcGetErrorString", &n.error_string);
    if (!ok) {
      n.why = "NVRTC library lacks an expected entry point";
      return;
    }
    n.version(&n.major, &n.minor);
    n.ok = true;
  });
  return n;
}

// 64-bit FNV-1a
uint64_t fnv1a(const std::string& s, uint64_t h = 1469598103934665603ull) {
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

std::string hexf(double v) {
  char b[64];
  snprintf(b, sizeof b, "%a", v);
  return b;
}

// The launch shape's body and geometry, after the same fall-backs the
// ahead-of-time dispatch applies.
struct Shape {
  const char* body;  // device function in bssn_kernels.cuh
  int tx, ty, minb;
  int xshare;        // 0 direct, 1 x lanes, 2 x lanes + y through shared memory
};

Shape shape_of(const Dims& d, int variant) {
  const LaunchVariant* v = variant_info(CHEMORA_BSSN, variant);
  if (!v || (v->xshare && (d.nx % v->tx != 0 || d.g < 3)))
    v = variant_info(CHEMORA_BSSN, 0);
  static const char* const bodies[] = {"bssn_direct_body", "bssn_x_body", "bssn_xy_body"};
  return Shape{bodies[v->xshare], v->tx, v->ty, v->minb, v->xshare};
}

std::string kernel_source(const Dims& d, const Scalars& sc, const Shape& sh, int mode) {
  char b[4096];
  std::string src = "// run-time specialised BSSN stage kernel\n#include \"bssn_kernels.cuh\"\n";
  snprintf(b, sizeof b,
           "struct JitScalars {\n"
           "  static constexpr double i12h = %s, i12h2 = %s, i144h2 = %s, ko_scale = %s, eta = %s;\n"
           "  static constexpr double ih = %s, ih2 = %s;\n"
           "  static constexpr int slicing = %d, shift = %d, order = %d;\n"
           "  double k[CHEMORA_NK];  // constant table: a kernel parameter, never folded\n"
           "};\n",
           hexf(sc.i12h).c_str(), hexf(sc.i12h2).c_str(), hexf(sc.i144h2).c_str(),
           hexf(sc.ko_scale).c_str(), hexf(sc.eta).c_str(), hexf(sc.ih).c_str(), hexf(sc.ih2).c_str(),
           sc.slicing, sc.shift, sc.order);
  src += b;
  snprintf(b, sizeof b,
           "extern \"C\" __global__ void __launch_bounds__(%d, %d)\n"
           "chemora_jit_stage(chemora::StageParams a0, chemora::KTable kt) {\n"
           "  const chemora::Dims d = {%d, %d, %d, %d, %lldLL, %lldLL, %lldLL};\n"
           "  chemora::StageParams a = a0;\n"
           "  a.mode = %d;\n"
           "  JitScalars sc;\n"
           "#pragma unroll\n"
           "  for (int q = 0; q < CHEMORA_NK; ++q) sc.k[q] = kt.k[q];\n",
           sh.tx * sh.ty, sh.minb, d.nx, d.ny, d.nz, d.g, (long long)d.sy, (long long)d.sz,
           (long long)d.sv, mode);
  src += b;
  if (sh.xshare == 2) {
    snprintf(b, sizeof b,
             "  extern __shared__ double smem[];\n"
             "  chemora::%s<%d, %d>(d, sc, a, smem);\n}\n",
             sh.body, sh.tx, sh.ty);
  } else {
    snprintf(b, sizeof b, "  chemora::%s<%d, %d>(d, sc, a);\n}\n", sh.body, sh.tx, sh.ty);
  }
  src += b;
  return src;
}

std::string default_cache_dir() {
  const char* e = getenv("CHEMORA_JIT_CACHE");
  if (e) return e;  // empty: no disk cache
  const char* home = getenv("HOME");
  if (!home || !*home) return "";
  return std::string(home) + "/.cache/chemora_jit";
}

bool make_dirs(const std::string& dir) {
  if (dir.empty()) return false;
  std::string cur;
  size_t pos = 0;
  while (pos != std::string::npos) {
    pos = dir.find('/', pos + 1);
    cur = dir.substr(0, pos);
    if (!cur.empty()) mkdir(cur.c_str(), 0755);
  }
  struct stat st;
  return stat(dir.c_str(), &st) == 0 && S_ISDIR(st.st_mode);
}

bool read_file(const std::string& path, std::vector<char>* out) {
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return false;
  std::vector<char> buf;
  char tmp[65536];
  size_t n;
  while ((n = fread(tmp, 1, sizeof tmp, f)) > 0) buf.insert(buf.end(), tmp, tmp + n);
  fclose(f);
  // an ELF64 header (64 bytes) for machine EM_CUDA (190), else not a cubin
  if (buf.size() < 64 || memcmp(buf.data(), "\x7f" "ELF", 4) != 0 || buf[4] != 2 ||
      ((unsigned char)buf[18] | ((unsigned char)buf[19] << 8)) != 190)
    return false;
  *out = std::move(buf);
  return true;
}

void write_file(const std::string& path, const std::vector<char>& data) {
  const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return;
  const bool ok = fwrite(data.data(), 1, data.size(), f) == data.size();
  if (fclose(f) == 0 && ok)
    rename(tmp.c_str(), path.c_str());
  else
    unlink(tmp.c_str());
}

struct CompileJob {
  std::string src, cache_file;
  std::vector<char> cubin;
  bool cached = false;
  std::string error;
};

void compile_one(const Nvrtc& n, const std::vector<std::string>& opts, CompileJob* job) {
  if (!job->cache_file.empty() && read_file(job->cache_file, &job->cubin)) {
    job->cached = true;
    return;
  }
  std::vector<std::string> texts(kNumJitHeaders);
  std::vector<const char*> hdr(kNumJitHeaders), names(kNumJitHeaders);
  for (int h = 0; h < kNumJitHeaders; ++h) {
    for (int c = 0; c < kJitHeaders[h].nchunks; ++c) texts[h] += kJitHeaders[h].chunks[c];
    hdr[h] = texts[h].c_str();
    names[h] = kJitHeaders[h].name;
  }
  nvrtcProgram prog;
  nvrtcResult r = n.create(&prog, job->src.c_str(), "chemora_jit_stage.cu", kNumJitHeaders, hdr.data(),
                           names.data());
  if (r != NVRTC_SUCCESS) {
    job->error = std::string("nvrtcCreateProgram: ") + n.error_string(r);
    return;
  }
  std::vector<const char*> o;
  for (const std::string& s : opts) o.push_back(s.c_str());
  r = n.compile(prog, (int)o.size(), o.data());
  if (r != NVRTC_SUCCESS) {
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) n.log(prog, &log[0]);
    if (log.size() > 1500) log.resize(1500);
    job->error = std::string("nvrtcCompileProgram: ") + n.error_string(r) + ": " + log;
    n.destroy(&prog);
    return;
  }
  if (getenv("CHEMORA_JIT_VERBOSE")) {  // the assembler's resource report
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) n.log(prog, &log[0]);
    fprintf(stderr, "chemora jit: %s", log.c_str());
  }
  size_t cs = 0;
  n.cubin_size(prog, &cs);
  job->cubin.resize(cs);
  if (cs) n.cubin(prog, job->cubin.data());
  n.destroy(&prog);
  if (cs == 0) {
    job->error = "NVRTC produced no cubin";
    return;
  }
  if (!job->cache_file.empty()) write_file(job->cache_file, job->cubin);
}

}  // namespace

struct JitModule {
  int variant = -1;
  dim3 grid, block;
  unsigned smem = 0;
  cudaLibrary_t lib[kModes] = {};
  cudaKernel_t k[kModes] = {};
  double compile_s = 0.0;
  int cached = 0;
};

void jit_free(chemora_system* sys) {
  if (!sys->jit) return;
  for (int m = 0; m < kModes; ++m)
    if (sys->jit->lib[m]) cudaLibraryUnload(sys->jit->lib[m]);
  delete sys->jit;
  sys->jit = nullptr;
  sys->jit_on = 0;
}

bool jit_active(const chemora_system* sys) {
  return sys->jit_on && sys->jit && sys->jit->variant == sys->variant;
}

int jit_launch(chemora_system* sys, const StageParams& a, cudaStream_t s) {
  const JitModule* J = sys->jit;
  if (a.mode < 0 || a.mode >= kModes) return set_error(CHEMORA_EINVAL, "stage mode %d", a.mode);
  StageParams p = a;
  KTable kt;
  for (int i = 0; i < CHEMORA_NK; ++i) kt.k[i] = sys->sc.k[i];
  void* args[] = {&p, &kt};
  CHEMORA_CUDA(cudaLaunchKernel((const void*)J->k[a.mode], J->grid, J->block, args, J->smem, s));
  return launched("chemora_jit_stage");
}

static int jit_build(chemora_system* sys, const char* cache_dir) {
  const Nvrtc& n = nvrtc();
  if (!n.ok) return set_error(CHEMORA_EUNSUPPORTED, "run-time specialisation: %s", n.why.c_str());
  const Dims& d = sys->grid->d;
  const Shape sh = shape_of(d, sys->variant);
  // target: the device's architecture (the ahead-of-time kernels are sm_103a)
  int major = 10, minor = 3, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  } else {
    cudaGetLastError();
  }
  char arch[64];
  snprintf(arch, sizeof arch, "--gpu-architecture=sm_%d%da", major, minor);
  std::vector<std::string> opts = {arch, "--std=c++17", "-DCHEMORA_JIT=1", "--fmad=true"};
  if (getenv("CHEMORA_JIT_VERBOSE")) opts.push_back("--ptxas-options=-v");
  std::string dir = cache_dir ? cache_dir : default_cache_dir();
  const bool use_cache = make_dirs(dir);
  std::vector<CompileJob> jobs(kModes);
  // the key covers the compiler version, the options and every embedded
  // header (a rebuilt library with other kernel bodies must not load cubins
  // compiled from the old ones)
  std::string key = std::to_string(n.major) + "." + std::to_string(n.minor);
  for (const std::string& o : opts) key += "|" + o;
  uint64_t hh = fnv1a(key);
  for (int h = 0; h < kNumJitHeaders; ++h) {
    hh = fnv1a(kJitHeaders[h].name, hh);
    for (int c = 0; c < kJitHeaders[h].nchunks; ++c) hh = fnv1a(kJitHeaders[h].chunks[c], hh);
  }
  for (int m = 0; m < kModes; ++m) {
    jobs[m].src = kernel_source(d, sys->sc, sh, m);
    if (use_cache) {
      char f[64];
      snprintf(f, sizeof f, "/stage_%016llx.cubin", (unsigned long long)fnv1a(jobs[m].src, hh));
      jobs[m].cache_file = dir + f;
    }
  }
  const auto t0 = std::chrono::steady_clock::now();
  {
    std::vector<std::thread> th;
    for (int m = 0; m < kModes; ++m) th.emplace_back(compile_one, std::cref(n), std::cref(opts), &jobs[m]);
    for (auto& t : th) t.join();
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (const CompileJob& j : jobs)
    if (!j.error.empty()) return set_error(CHEMORA_ECUDA, "run-time specialisation: %s", j.error.c_str());
  JitModule* J = new (std::nothrow) JitModule();
  if (!J) return set_error(CHEMORA_ENOMEM, "host allocation");
  J->variant = sys->variant;
  J->block = dim3(sh.tx, sh.ty, 1);
  // the grids of the ahead-of-time launchers in bssn.cu
  J->grid = dim3(sh.xshare == 0 ? (d.nx + sh.tx - 1) / sh.tx : d.nx / sh.tx, (d.ny + sh.ty - 1) / sh.ty, d.nz);
  J->smem = sh.xshare == 2 ? bssn_xy_smem_bytes(sh.tx, sh.ty) : 0u;
  J->compile_s = secs;
  J->cached = 1;
  for (const CompileJob& j : jobs) J->cached &= j.cached ? 1 : 0;
  int rc = CHEMORA_OK;
  for (int m = 0; m < kModes && !rc; ++m) {
    cudaError_t e = cudaLibraryLoadData(&J->lib[m], jobs[m].cubin.data(), nullptr, nullptr, 0, nullptr,
                                        nullptr, 0);
    if (e != cudaSuccess && jobs[m].cached) {
      // a damaged cache entry: compile afresh (and overwrite it) once
      cudaGetLastError();
      jobs[m].cached = false;
      jobs[m].cubin.clear();
      const std::string file = jobs[m].cache_file;
      unlink(file.c_str());
      compile_one(n, opts, &jobs[m]);
      if (!jobs[m].error.empty()) {
        rc = set_error(CHEMORA_ECUDA, "run-time specialisation: %s", jobs[m].error.c_str());
        break;
      }
      J->cached = 0;
      e = cudaLibraryLoadData(&J->lib[m], jobs[m].cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    }
    if (e != cudaSuccess) {
      J->lib[m] = nullptr;
      rc = cuda_error(e, "cudaLibraryLoadData (specialised stage kernel)");
      break;
    }
    e = cudaLibraryGetKernel(&J->k[m], J->lib[m], "chemora_jit_stage");
    if (e == cudaSuccess && J->smem)
      e = cudaFuncSetAttribute((const void*)J->k[m], cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)J->smem);
    if (e != cudaSuccess) rc = cuda_error(e, "cudaLibraryGetKernel (specialised stage kernel)");
  }
  jit_free(sys);
  sys->jit = J;
  if (rc) {
    jit_free(sys);
    return rc;
  }
  return CHEMORA_OK;
}

}  // namespace chemora

using namespace chemora;

extern "C" {

int chemora_system_specialize(chemora_system* sys, int enable, const char* cache_dir,
                              double* compile_seconds) {
  if (!is_handle(sys, H_SYSTEM)) return set_error(CHEMORA_EINVAL, "not a system handle");
  if (compile_seconds) *compile_seconds = 0.0;
  free_step_graph(sys);
  if (!enable) {
    sys->jit_on = 0;
    return CHEMORA_OK;
  }
  if (sys->kind != CHEMORA_BSSN)
    return set_error(CHEMORA_EUNSUPPORTED, "run-time specialisation is built for BSSN systems only");
  if (!(sys->jit && sys->jit->variant == sys->variant)) {
    int rc = jit_build(sys, cache_dir);
    if (rc) return rc;
    if (compile_seconds) *compile_seconds = sys->jit->cached ? 0.0 : sys->jit->compile_s;
  }
  sys->jit_on = 1;
  return CHEMORA_OK;
}

}  // extern "C"
