"""Build libspock.so in-tree with nvcc for sm_103a.

    python -m paper_2505_12078_b300.build          # build (skips if up to date)
    python -m paper_2505_12078_b300.build --force
    python -m paper_2505_12078_b300.build -v       # print ptxas register/spill report

libspock_checked.so is the same library compiled with -DSPOCK_CHECKED (index
checks in the iteration kernel, see spock_debug_last_check).

Every translation unit (and every solver kernel variant) is compiled to an
object in parallel, then linked into one shared library.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
OUT = os.path.join(HERE, "libspock.so")
# the bounds-checked variant (-DSPOCK_CHECKED: index checks in the iteration kernel)
OUT_CHECKED = os.path.join(HERE, "libspock_checked.so")
HEADERS = ["spock_dev.cuh", "spock_internal.h", "spock_solver_kernel.cuh", "spock_cta.cuh", "spock_problem.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (object name, source, extra defines)
UNITS = [
    ("spock_api", "spock_api.cu", []),
    ("spock_setup", "spock_setup.cu", []),
    ("spock_setup_ext", "spock_setup_ext.cu", []),
    ("spock_solver", "spock_solver.cu", []),
    ("spock_noalloc", "spock_noalloc.cu", []),
    ("spock_diag", "spock_diag.cu", []),
    ("spock_centre", "spock_centre.cu", []),
    ("spock_batch", "spock_batch.cu", []),
    ("spock_serve", "spock_serve.cu", []),
    ("solver_f1", "spock_solver_inst.cu", ["-DSPOCK_T=float", "-DSPOCK_CH=1", "-DSPOCK_SUFFIX=f1", "-DSPOCK_WITH_BATCH"]),
    ("solver_f2", "spock_solver_inst.cu", ["-DSPOCK_T=float", "-DSPOCK_CH=2", "-DSPOCK_SUFFIX=f2"]),
    ("solver_d2", "spock_solver_inst.cu", ["-DSPOCK_T=double", "-DSPOCK_CH=2", "-DSPOCK_SUFFIX=d2", "-DSPOCK_WITH_BATCH"]),
    ("solver_d4", "spock_solver_inst.cu", ["-DSPOCK_T=double", "-DSPOCK_CH=4", "-DSPOCK_SUFFIX=d4"]),
]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *ARCH]


def nvcc():
    c = os.environ.get("NVCC")
    if c:
        return c
    if os.path.exists("/usr/local/cuda/bin/nvcc"):
        return "/usr/local/cuda/bin/nvcc"
    return "nvcc"


def _deps(src):
    d = [os.path.join(CSRC, src)] + [os.path.join(CSRC, h) for h in HEADERS]
    d.append(os.path.join(HERE, "..", "include", "spock.h"))
    d.append(os.path.abspath(__file__))
    return [x for x in d if os.path.exists(x)]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(unit, verbose, tag=""):
    name, src, defs = unit
    obj = os.path.join(OBJ, name + tag + ".o")
    cmd = [nvcc(), "-c", *FLAGS, *defs, "-o", obj + ".tmp", os.path.join(CSRC, src)]
    if verbose:
        cmd[2:2] = ["-Xptxas", "-v"]
    r = subprocess.run(cmd, cwd=CSRC, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {name}:\n{r.stdout}{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return name, r.stderr


def _build_one(out, units, tag, force, verbose):
    todo = [u for u in units
            if force or _stale(os.path.join(OBJ, u[0] + tag + ".o"), _deps(u[1]))]
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            for name, log in ex.map(lambda u: _compile(u, verbose, tag), todo):
                if verbose:
                    sys.stderr.write(f"== {name}{tag}\n{log}")
    objs = [os.path.join(OBJ, u[0] + tag + ".o") for u in units]
    if todo or force or _stale(out, objs):
        cmd = [nvcc(), "-shared", *ARCH, "-o", out + ".tmp", *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stdout}{r.stderr}")
        os.replace(out + ".tmp", out)
    return out


def build(force=False, verbose=False, checked=True):
    """Builds libspock.so and (checked=True) the bounds-checked libspock_checked.so."""
    os.makedirs(OBJ, exist_ok=True)
    _build_one(OUT, UNITS, "", force, verbose)
    if checked:
        _build_one(OUT_CHECKED, [(n, src, d + ["-DSPOCK_CHECKED"]) for (n, src, d) in UNITS], "_chk", force, verbose)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(OUT)
