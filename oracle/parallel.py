"""The oracle's TOD on several host cores.  ORACLE: test and benchmark infrastructure only.

No arithmetic of the method lives here: each worker is a fresh single-threaded
interpreter (``python -m oracle.parallel``, started by fork+exec, so it is safe
to call from a process that already holds a CUDA context) that runs
``oracle.convolve.tod`` one sample at a time on consecutive samples from its
own start offset until its time budget is spent.  The inputs reach the workers
as ``.npy`` files in a temporary folder (the sky memory-mapped, so the page
cache holds one copy); the loops start together, once every worker has loaded
them and run one untimed warm-up sample, and each worker writes back its outputs and the wall clock at the start
and end of its loop.  The aggregate rate is the samples of all workers over the
span from the first start to the last end, which excludes interpreter start-up
but includes any imbalance between the workers.
"""

import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_ONE_THREAD = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}


def host_cores():
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def tod_sampled(nside, radius, sky, grids, det, omega, theta0, phi0, psi0, processes=None, budget_s=15.0,
                max_per_worker=None):
    """Run ``oracle.convolve.tod`` in ``processes`` workers for about ``budget_s`` seconds each.

    Worker j starts at sample j * n / processes and takes consecutive samples.
    Returns ``(index, d, span_s, processes)``: the sample indices processed
    (ascending), their TOD values, and the wall-clock span of the parallel loop.
    """
    n = len(theta0)
    processes = max(1, min(processes or host_cores(), n))
    limit = max_per_worker if max_per_worker is not None else n
    with tempfile.TemporaryDirectory(prefix="oracle_tod_") as tmp:
        for name, a in (("sky", sky), ("grids", grids), ("theta", theta0), ("phi", phi0), ("psi", psi0)):
            np.save(os.path.join(tmp, name + ".npy"), np.ascontiguousarray(a, np.float64))
        with open(os.path.join(tmp, "job.json"), "w") as f:
            json.dump({"nside": int(nside), "radius": float(radius), "det": [float(x) for x in det],
                       "omega": [float(x) for x in np.atleast_1d(omega)], "budget_s": float(budget_s)}, f)
        env = dict(os.environ, **_ONE_THREAD)
        env["PYTHONPATH"] = _ROOT + os.pathsep + env.get("PYTHONPATH", "")
        procs = []
        try:
            for j in range(processes):
                a = n * j // processes
                b = min(n * (j + 1) // processes, a + limit)
                procs.append(subprocess.Popen(
                    [sys.executable, "-m", "oracle.parallel", tmp, str(j), str(a), str(b)], cwd=_ROOT, env=env))
            # start the loops together once every worker has loaded its inputs
            deadline = time.time() + 600.0
            while not all(os.path.exists(os.path.join(tmp, f"ready{j}")) for j in range(processes)):
                if time.time() > deadline or any(p.poll() not in (None, 0) for p in procs):
                    raise RuntimeError("oracle workers did not start")
                time.sleep(0.002)
            open(os.path.join(tmp, "go"), "w").close()
            codes = [p.wait() for p in procs]
        finally:
            for p in procs:  # none is left running when this call ends, however it ends
                if p.poll() is None:
                    p.kill()
                    p.wait()
        if any(codes):
            raise RuntimeError(f"oracle workers failed with exit codes {codes}")
        idx, vals, t0, t1 = [], [], [], []
        for j in range(processes):
            with open(os.path.join(tmp, f"w{j}.json")) as f:
                info = json.load(f)
            t0.append(info["t0"])
            t1.append(info["t1"])
            idx.append(np.arange(info["a"], info["a"] + info["k"]))
            vals.append(np.load(os.path.join(tmp, f"w{j}.npy")))
    return np.concatenate(idx), np.concatenate(vals), max(t1) - min(t0), processes


def _worker(tmp, j, a, b):
    from . import convolve as oc
    with open(os.path.join(tmp, "job.json")) as f:
        job = json.load(f)
    sky = np.load(os.path.join(tmp, "sky.npy"), mmap_mode="r")
    grids = np.load(os.path.join(tmp, "grids.npy"))
    th, ph, ps = (np.load(os.path.join(tmp, k + ".npy"), mmap_mode="r") for k in ("theta", "phi", "psi"))
    omega = np.asarray(job["omega"], np.float64)
    omega = omega[0] if omega.size == 1 else omega

    def one(k):
        return oc.tod(job["nside"], job["radius"], sky, grids, tuple(job["det"]), omega, th[k:k + 1], ph[k:k + 1],
                      ps[k:k + 1])[0]

    if a < b:
        one(a)  # untimed warm-up: first-touch of the inputs and of numpy's code paths
    open(os.path.join(tmp, f"ready{j}"), "w").close()
    deadline = time.time() + 600.0
    while not os.path.exists(os.path.join(tmp, "go")):
        if time.time() > deadline:
            raise SystemExit("no start signal")
        time.sleep(0.0005)
    out = []
    t0 = time.time()
    k = a
    while k < b and time.time() - t0 < job["budget_s"]:
        out.append(one(k))
        k += 1
    t1 = time.time()
    np.save(os.path.join(tmp, f"w{j}.npy"), np.asarray(out, np.float64))
    with open(os.path.join(tmp, f"w{j}.json"), "w") as f:
        json.dump({"a": a, "k": k - a, "t0": t0, "t1": t1}, f)


if __name__ == "__main__":
    _worker(sys.argv[1], int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]))
