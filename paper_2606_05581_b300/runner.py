"""Checkpointed batched estimates over many meshes (host-side orchestration).

Large sweeps (the paper's per-shape preprocessing of hundreds of thousands of
meshes, Sec. 6) run as chunks of meshes through the batched estimate
(mcs_estimate_batched: one persistent walk launch per chunk).  Every mesh's
outputs are written to its own file in ``out_dir`` as soon as its chunk
finishes, through a temporary file that is flushed to disk and renamed into
place, so a file that exists is complete.  A rerun with the same directory
skips the meshes whose files exist.  A mesh's outputs depend only on its
geometry, its rows, the parameters, its domain and its seed (counter-based
walks, exact closest points): never on which other meshes share its chunk, so
a resumed sweep reproduces an uninterrupted one bit for bit.

Nothing here computes any part of the estimate: the chunk's work is done by
the ``estimate`` callable, by default the library's batched GPU estimate.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Callable, Iterable

import numpy as np

MANIFEST = "manifest.json"
# per-mesh arrays written to each file (when present)
ARRAYS = ("hist_ptr", "hist_bin", "hist_cnt", "omega", "H0", "Lambda", "evals", "evecs", "row_pos", "row_nrm",
          "row_area")


def mesh_file(out_dir: str, mesh_id: int) -> str:
    return os.path.join(out_dir, f"mesh_{mesh_id:07d}.npz")


def params_digest(params: dict) -> str:
    """A digest of the sweep's settings; a resume with other settings is refused."""
    return hashlib.sha256(json.dumps(params, sort_keys=True).encode()).hexdigest()[:32]


def done_ids(out_dir: str) -> set:
    out = set()
    if not os.path.isdir(out_dir):
        return out
    for name in os.listdir(out_dir):
        if name.startswith("mesh_") and name.endswith(".npz"):
            out.add(int(name[5:-4]))
    return out


def write_atomic(path: str, arrays: dict, meta: dict) -> None:
    """Write one mesh's outputs: temporary file, flush + fsync, rename."""
    d = os.path.dirname(path)
    tmp = os.path.join(d, "." + os.path.basename(path) + f".{os.getpid()}.tmp")
    with open(tmp, "wb") as fh:
        np.savez(fh, meta=np.frombuffer(json.dumps(meta, sort_keys=True).encode(), dtype=np.uint8), **arrays)
        fh.flush()
        os.fsync(fh.fileno())
    os.replace(tmp, path)
    try:  # make the rename itself durable
        fd = os.open(d, os.O_RDONLY)
        try:
            os.fsync(fd)
        finally:
            os.close(fd)
    except OSError:
        pass


def read_mesh(out_dir: str, mesh_id: int) -> tuple:
    """(arrays, meta) of a written mesh."""
    with np.load(mesh_file(out_dir, mesh_id)) as z:
        arrays = {k: z[k] for k in z.files if k != "meta"}
        meta = json.loads(bytes(z["meta"]).decode())
    return arrays, meta


def _open_sweep(out_dir: str, settings: dict) -> None:
    """Create or check the directory's manifest; one sweep writes a directory
    at a time, so temporary files found here are leftovers of an interrupted
    write (never complete results) and are removed."""
    os.makedirs(out_dir, exist_ok=True)
    path = os.path.join(out_dir, MANIFEST)
    digest = params_digest(settings)
    if os.path.exists(path):
        with open(path) as fh:
            old = json.load(fh)
        if old.get("digest") != digest:
            raise ValueError(f"{out_dir} holds a sweep with other settings ({old.get('settings')}); "
                             "use another directory")
    else:
        write_json = json.dumps({"digest": digest, "settings": settings}, sort_keys=True, indent=1)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            fh.write(write_json)
            fh.flush()
            os.fsync(fh.fileno())
        os.replace(tmp, path)
    for name in os.listdir(out_dir):
        if name.startswith(".mesh_") and name.endswith(".tmp"):
            os.remove(os.path.join(out_dir, name))


def run_sweep(mesh_ids: Iterable[int], out_dir: str, estimate: Callable, settings: dict, chunk: int = 64,
              on_written: Callable | None = None) -> dict:
    """Estimate every mesh id not yet written under out_dir, ``chunk`` meshes
    per call of ``estimate(ids) -> list of (arrays, meta)`` (one per id, in
    order), writing each mesh's file as its chunk returns.  ``settings`` (a
    JSON-able dict) must match the directory's manifest on a resume.
    on_written(mesh_id) is called after each file is in place.  Returns
    counts of skipped and written meshes."""
    ids = [int(i) for i in mesh_ids]
    _open_sweep(out_dir, settings)
    have = done_ids(out_dir)
    todo = [i for i in ids if i not in have]
    written = 0
    for c in range(0, len(todo), chunk):
        part = todo[c:c + chunk]
        results = estimate(part)
        if len(results) != len(part):
            raise RuntimeError("estimate returned a different number of meshes than it was given")
        for mid, (arrays, meta) in zip(part, results):
            meta = dict(meta, mesh_id=mid, settings_digest=params_digest(settings))
            write_atomic(mesh_file(out_dir, mid), {k: v for k, v in arrays.items() if v is not None}, meta)
            written += 1
            if on_written is not None:
                on_written(mid)
    return {"requested": len(ids), "skipped": len(ids) - len(todo), "written": written}


def gpu_estimate(make_mesh: Callable, rows_per_mesh: int, params, domain_of: Callable = lambda i: i % 2,
                 seed_of: Callable = lambda i: i, keep_lambda: bool = False, k: int = 0) -> Callable:
    """The default chunk estimate: the meshes' BVHs and farthest-point sample
    rows, one batched estimate (one persistent walk launch), and optionally
    each mesh's k smallest Steklov pairs, copied to host arrays."""
    import torch

    from . import Batch, build_meshes, sample_rows_batched, steklov_modes

    def estimate(ids):
        hosts = [make_mesh(i) for i in ids]
        meshes = build_meshes([(h.V, h.F) for h in hosts])
        rows = sample_rows_batched(meshes, rows_per_mesh, orient=True)
        items = [dict(mesh=m, rows={q: r[q] for q in ("pos", "nrm", "area", "tri2bin")}, domain=int(domain_of(i)),
                      seed=int(seed_of(i))) for i, m, r in zip(ids, meshes, rows)]
        b = Batch(items, params, assemble=keep_lambda or k > 0)
        _, _, per = b.run()
        out = []
        for j, i in enumerate(ids):
            res = b.result(j)
            # the padded CSR compacted: row v's (bin, count) pairs at hist_ptr[v] .. hist_ptr[v + 1]
            nnz = res["hist_nnz"].cpu().numpy().astype(np.int64)
            cap = int(res["cap"])
            filled = (np.arange(cap)[None, :] < nnz[:, None]).ravel()
            arrays = {"hist_ptr": np.concatenate([[0], np.cumsum(nnz)]).astype(np.int64),
                      "hist_bin": res["hist_bin"].cpu().numpy()[filled],
                      "hist_cnt": res["hist_cnt"].cpu().numpy()[filled]}
            arrays.update({q: res[q].cpu().numpy() for q in ("omega", "H0") if res.get(q) is not None})
            arrays.update(row_pos=rows[j]["pos"].cpu().numpy(), row_nrm=rows[j]["nrm"].cpu().numpy(),
                          row_area=rows[j]["area"].cpu().numpy())
            if k > 0:
                ev, X, _ = steklov_modes(res["Lambda"], rows[j]["area"], k)
                arrays.update(evals=ev.cpu().numpy(), evecs=X.cpu().numpy())
            if keep_lambda:
                arrays["Lambda"] = res["Lambda"].cpu().numpy()
            st = {q: per[j][q] for q in ("walks", "steps", "capped", "lost", "discarded_rows", "killing_steps")}
            out.append((arrays, dict(stats=st, domain=int(domain_of(i)), seed=int(seed_of(i)),
                                     faces=int(hosts[j].nf), rows=rows_per_mesh)))
        torch.cuda.synchronize()
        return out

    return estimate


def main():
    import argparse
    import sys

    ap = argparse.ArgumentParser(description="checkpointed batched estimates of the synthetic mesh batch")
    ap.add_argument("--out", required=True)
    ap.add_argument("--meshes", type=int, default=512)
    ap.add_argument("--chunk", type=int, default=64)
    ap.add_argument("--rows", type=int, default=1024)
    ap.add_argument("--walks", type=int, default=512)
    ap.add_argument("--k", type=int, default=0, help="Steklov pairs per mesh (0: none)")
    a = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import meshgen

    from . import default_params
    p = default_params(walks_per_row=a.walks, killing_walks=64 * a.walks)
    settings = dict(workload="batch meshes seed 1000 + i", rows=a.rows, walks=a.walks, killing_walks=64 * a.walks,
                    k=a.k, domain="exterior for odd i", seed="i")
    est = gpu_estimate(meshgen.batch_mesh, a.rows, p, k=a.k)
    print(json.dumps(run_sweep(range(a.meshes), a.out, est, settings, chunk=a.chunk)))


if __name__ == "__main__":
    main()
