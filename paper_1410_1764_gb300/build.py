"""Build libchemora.so (sm_103a) in-tree with nvcc.

Each .cu under csrc/ is compiled to an object in parallel, then linked into
paper_1410_1764_gb300/libchemora.so.  The generated point bodies under
csrc/generated/ are committed sources; the one file written here is
csrc/generated/jit_sources.inc, the device headers the run-time specialiser
(csrc/jit.cu) hands to NVRTC, embedded as string literals.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libchemora.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC]


# device headers the run-time specialised stage kernel includes (NVRTC)
JIT_HEADERS = ("device_types.cuh", "stage.cuh", "bssn_kernels.cuh", "generated/gen_constants.cuh",
               "generated/gen_bssn.cuh", "generated/gen_bssn_x.cuh", "generated/gen_bssn_xy.cuh")
JIT_INC = os.path.join(CSRC, "generated", "jit_sources.inc")
_DELIM = "chemora_src"
_CHUNK = 12000


def write_jit_sources():
    """Write csrc/generated/jit_sources.inc (only when its text changes)."""
    out = ["// WRITTEN by paper_1410_1764_gb300/build.py from the headers it names; do not edit.\n"]
    entries = []
    for h, rel in enumerate(JIT_HEADERS):
        with open(os.path.join(CSRC, rel)) as f:
            text = f.read()
        if (")" + _DELIM + '"') in text:
            raise RuntimeError("%s contains the raw-string delimiter" % rel)
        chunks = [text[i:i + _CHUNK] for i in range(0, len(text), _CHUNK)] or [""]
        out.append("static const char* const kJitChunks%d[] = {\n" % h)
        for c in chunks:
            out.append('R"%s(%s)%s",\n' % (_DELIM, c, _DELIM))
        out.append("};\n")
        entries.append('    {"%s", kJitChunks%d, %d},\n' % (rel, h, len(chunks)))
    out.append("static const JitHeader kJitHeaders[] = {\n" + "".join(entries) + "};\n")
    out.append("static const int kNumJitHeaders = %d;\n" % len(JIT_HEADERS))
    text = "".join(out)
    old = None
    if os.path.exists(JIT_INC):
        with open(JIT_INC) as f:
            old = f.read()
    if old != text:
        with open(JIT_INC, "w") as f:
            f.write(text)


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    out = []
    for d in (CSRC, os.path.join(CSRC, "generated"), os.path.join(ROOT, "include")):
        out += [os.path.join(d, f) for f in os.listdir(d)
                if f.endswith((".h", ".cuh", ".inc"))]
    return out


def _stale(obj, src, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + deps)


def build(force=False, verbose=False):
    os.makedirs(OBJ, exist_ok=True)
    write_jit_sources()
    nvcc = _nvcc()
    deps = _deps()
    jobs = []
    for src in sources():
        obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, src, deps):
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append((src, cmd))
    objs = [os.path.join(OBJ, os.path.basename(s)[:-3] + ".o") for s in sources()]

    def run(job):
        src, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r

    failed = []
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        for src, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for: %s" % ", ".join(failed))
    if jobs or force or not os.path.exists(LIB) or any(
            os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
