"""The device code of the per-track fit compiled for the host CPU (test and study tool).

`build()` copies the device headers of the package (kf_common.cuh, kf_track.cuh,
kf_df.cuh, kf_internal.h) and the device-side sections of kf_fit.cu (the seed-hit
helpers and the fit: fit_step, the crossing kinds, the out-of-line steps,
fit_phase1/2, fit_track) into tests/_build/host_replica/, with one substitution
(the FP64 reciprocal approximation, inline PTX, becomes an FP32 reciprocal), and
compiles them with host definitions of the CUDA intrinsics
(tests/host_replica/host_fit.cpp) into a shared library.  `host_fit()` fits
tracks with it, one at a time, on the host.

It lets the arithmetic of the kernels be studied against the oracle on a CPU: the
precision readings of the mixed fit were measured with it (a step of the fit
replaced in the copy, then the parity of the result), and
tests/test_host_replica.py keeps the copy itself at the tolerances.  The library
never runs it.
"""
import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1711_06571_gb300", "csrc")
OUT = os.path.join(HERE, "_build", "host_replica")
FIT_SECTIONS = (("template <bool B, class X, class Y> struct sel", "__global__ void __launch_bounds__(128) seed_kernel"),
                ("// ------------------------------------------------------------------ fit",
                 "// ------------------------------------------------------------------ the mixed fit in two kernels"))
RCP_PTX = 'asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));'


def assemble(out=OUT, edit=None):
    """Write the host copy of the sources into `out`.  edit: optional function
    (file name, text) -> text applied to each copied file (for studies)."""
    os.makedirs(out, exist_ok=True)
    edit = edit or (lambda name, text: text)
    s = open(os.path.join(CSRC, "kf_common.cuh")).read()
    if s.count(RCP_PTX) != 2:
        raise RuntimeError("kf_common.cuh: the reciprocal approximation changed; update host_replica.py")
    s = s.replace(RCP_PTX, "y = (double)(1.0f / (float)d);")
    s = s.replace('#include "../../include/kf.h"', '#include "%s"' % os.path.join(ROOT, "include", "kf.h"))
    open(os.path.join(out, "kf_common.cuh"), "w").write(edit("kf_common.cuh", s))
    for f in ("kf_track.cuh", "kf_df.cuh", "kf_internal.h"):
        open(os.path.join(out, f), "w").write(edit(f, open(os.path.join(CSRC, f)).read()))
    s = open(os.path.join(CSRC, "kf_fit.cu")).read()
    body = ""
    for a, b in FIT_SECTIONS:
        if a not in s or b not in s:
            raise RuntimeError("kf_fit.cu: section markers changed; update host_replica.py")
        body += s[s.index(a):s.index(b)]
    body = body.replace("static __device__ __noinline__", "static __device__ __attribute__((noinline))")
    hdr = ('#pragma once\n#include "kf_df.cuh"\n#include "kf_internal.h"\nnamespace kfd {\n'
           'constexpr double PI_D_FIT = 3.14159265358979323846;\n' + body + "\n}  // namespace kfd\n")
    open(os.path.join(out, "fit_track.h"), "w").write(edit("fit_track.h", hdr))
    src = open(os.path.join(HERE, "host_replica", "host_fit.cpp")).read()
    open(os.path.join(out, "host_fit.cpp"), "w").write(src)
    return out


def build(out=OUT, edit=None, name="host_fit.so"):
    """Assemble and compile; returns the loaded library."""
    out = assemble(out, edit)
    so = os.path.join(out, name)
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-w", "-I", out, "-I", cuda_inc,
           "-o", so, os.path.join(out, "host_fit.cpp")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("host replica build failed:\n" + r.stderr[-4000:])
    lib = C.CDLL(so)
    return lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def host_fit(lib, geom, tk, seed, q, seed_df=1, n64=3, fp64=0, meas_model=0):
    """Fit the CSR tracks tk with the host copy: seed (n, 6) FP32 seeds, q (n,)
    charges.  Returns state (n, 6), cov (n, 6, 6), chi2, ndof, status, q."""
    sp = np.array([[s["kind"], s["pos"], s["half_or_rin"], s.get("r_out", 0.0), s["x_x0"], s["sig_n"],
                    s["sig_rphi"], s["sig_3"], s.get("dr", 0.0)] for s in geom["surfaces"]], np.float64)
    n = int(tk["n"])
    seed_t = np.ascontiguousarray(np.asarray(seed, np.float32).T)
    qq = np.ascontiguousarray(np.asarray(q, np.int8))
    off = np.ascontiguousarray(tk["offsets"], np.int32)
    lay = np.ascontiguousarray(tk["layer"], np.uint8)
    x, y, z = (np.ascontiguousarray(tk[k], np.float32) for k in "xyz")
    st = np.zeros((6, n))
    cov = np.zeros((21, n))
    chi2 = np.zeros(n)
    ndof = np.zeros(n, np.int32)
    status = np.zeros(n, np.uint32)
    lib.host_fit(len(sp), _p(sp), C.c_double(geom["bz"]), C.c_double(geom["mass"]), n, _p(off), _p(lay), _p(x), _p(y),
                 _p(z), _p(seed_t), _p(qq), int(seed_df), int(n64), int(fp64), int(meas_model), _p(st), _p(cov),
                 _p(chi2), _p(ndof), _p(status))
    C6 = np.zeros((n, 6, 6))
    k = 0
    for i in range(6):
        for j in range(i + 1):
            C6[:, i, j] = cov[k]
            C6[:, j, i] = cov[k]
            k += 1
    return dict(state=st.T.copy(), cov=C6, chi2=chi2, ndof=ndof, status=status, q=qq)


def _define_edit(defs):
    """An edit that sets `constexpr <type> NAME = value;` in the copied sources."""
    import re

    def edit(name, text):
        for k, v in defs.items():
            pat = re.compile(r"(constexpr\s+\w+\s+%s\s*=\s*)[^;]+;" % re.escape(k))
            text, n = pat.subn(lambda m: m.group(1) + v + ";", text)
        return text
    return edit


def main(argv=None):
    """Parity of the host copy against the oracle:
        python tests/host_replica.py --geometry lids --tracks 20000 [--define NAME=VALUE ...]
    prints the largest parameter, chi2 and covariance deviations (parity.summary)
    and the number of tracks beyond max(1e-3 sigma, 3 x the oracle's resolution).
    --define sets a constexpr constant of the copied sources (e.g.
    NEAR_TANGENT_SINE=0.85f)."""
    import argparse
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, HERE)
    import oracle
    import parity
    from paper_1711_06571_gb300 import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--geometry", default="barrel17")
    ap.add_argument("--tracks", type=int, default=20000)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--define", action="append", default=[])
    ap.add_argument("--threads", type=int, default=8)
    args = ap.parse_args(argv)
    defs = dict(d.split("=", 1) for d in args.define)
    tag = "_".join(f"{k}{v}" for k, v in defs.items()).replace(".", "p") or "default"
    lib = build(out=os.path.join(HERE, "_build", "host_replica_" + tag), edit=_define_edit(defs))
    g = synth.geometry(args.geometry)
    kw = dict(eta_max=2.5, min_hits=4) if args.geometry == "lids" else {}
    model = 1 if args.geometry == "barrel17s" else 0
    tk = synth.gen_tracks(g, args.tracks, synth.BASE_SEED + args.seed, **kw)
    o0 = oracle.fit(g, tk, threads=args.threads, meas_model=model)
    seed = o0["seed"].astype(np.float32)
    orc = oracle.fit(g, tk, seeds=seed.astype(np.float64), q=o0["q"], threads=args.threads, meas_model=model)
    host = host_fit(lib, g, tk, seed, orc["q"], meas_model=model)
    ok = ((orc["status"] & 7) == 0) & ((host["status"] & 7) == 0) & (host["ndof"] == orc["ndof"])
    kinds = np.array([g["surfaces"][s]["kind"] for s in parity.last_surface(tk, orc["ndof"])])
    noise = parity.oracle_self_noise(oracle, g, tk, orc, kinds, threads=args.threads)
    res = parity.compare_fits(host, orc, kinds, ok)
    beyond = int(np.sum(res["max_pull"] > np.maximum(parity.TOL_PARAM_SIGMA, 3.0 * noise[ok])))
    nst = int(np.sum((host["status"] & 7) != (orc["status"] & 7)))
    print(f"{args.geometry} {args.tracks} tracks {defs or ''}: status differences {nst}, "
          f"beyond the bound {beyond}; {parity.summary(res)}")


if __name__ == "__main__":
    main()
