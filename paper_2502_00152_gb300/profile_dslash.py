"""Run a few plain CG iterations on a benchmark lattice so that a profiler can
capture the Dslash kernels in the same launch configuration as the solve.

usage: python -m paper_2502_00152_gb300.profile_dslash [--config c4] [--iters 4]
                                                      [--sloppy 16] [--recon 18] [--mrhs K]
                                                      [--reliable 48]
Kernel order of one call: source preparation and initial residual (three FP64
Dslash launches), then per CG iteration the D_oe kernel, the fused D_eo + update
kernel and the direction update.
"""
import argparse

from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I


def write_traffic(report: str, config: str, key: str, out: str, command: str) -> None:
    """Per-output-site DRAM bytes of the D_oe (EpiXpay) and fused D_eo + update
    (EpiCG) Dslash launches in an ncu report of this driver, written with the
    hash of the Dslash sources they were taken on (the benchmark uses them only
    while that hash matches)."""
    import csv
    import io
    import json
    import subprocess

    from paper_2502_00152_gb300.build import dslash_source_hash

    txt = subprocess.run(["ncu", "-i", report, "--page", "raw", "--csv"], check=True, capture_output=True,
                         text=True).stdout
    rows = list(csv.reader(io.StringIO(txt)))
    hdr, data = rows[0], rows[2:]
    col = {n: hdr.index(n) for n in ("Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum")}
    units = rows[1]
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    dims = I.lattice_config(config)["dims"]
    dims_s = f"{dims[0]}^3x{dims[3]}"
    vh = I.volume(dims) // 2
    per_site = {}
    for r in data:
        name = r[col["Kernel Name"]]
        kind = "oe" if "EpiXpay" in name else ("eo" if "EpiCG" in name else None)
        if kind is None:
            continue
        b = sum(float(r[col[m]].replace(",", "")) * scale[units[col[m]]]
                for m in ("dram__bytes_read.sum", "dram__bytes_write.sum"))
        per_site.setdefault(f"{kind}_{key}", []).append(b / vh)
    doc = {"what": f"DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per output site of the sloppy "
                   f"Dslash kernels, from one ncu capture on the {dims_s} lattice (Vh = {vh}); traffic scales with "
                   f"the number of output sites, so the benchmark multiplies by its own Vh",
           "command": command, "kernel_source_hash": dslash_source_hash(),
           "dram_bytes_per_output_site": {k: round(sum(v) / len(v), 1) for k, v in per_site.items()}}
    with open(out, "w") as f:
        json.dump(doc, f, indent=1)
    print(json.dumps(doc["dram_bytes_per_output_site"]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c4")
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--sloppy", type=int, default=16)
    ap.add_argument("--recon", type=int, default=18)
    ap.add_argument("--tc", type=int, default=0, help="also run the tensor-core batched deflation with this many "
                                                     "random eigenvectors (24 right-hand sides)")
    ap.add_argument("--tc-prec", type=int, default=32, help="eigenvector storage for --tc: 32 or 15 (BF16)")
    ap.add_argument("--mrhs", type=int, default=0, help="instead solve this many Gaussian right-hand sides together "
                                                        "(batched operator) for --iters iterations")
    ap.add_argument("--reliable", type=int, default=64, choices=[64, 48],
                    help="reliable-update arithmetic (48: the double-float residual kernels run once, at the "
                         "forced final update)")
    ap.add_argument("--traffic-from", default=None, metavar="REPORT",
                    help="instead write profiles/dslash_traffic.json from an ncu report of this driver")
    ap.add_argument("--traffic-key", default="s16_r12", help="suffix of the keys written (sloppy bits, recon)")
    ap.add_argument("--traffic-command", default="", help="the ncu command that made the report (recorded)")
    a = ap.parse_args()
    if a.traffic_from:
        import os

        out = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles",
                           "dslash_traffic.json")
        write_traffic(a.traffic_from, a.config, a.traffic_key, out, a.traffic_command)
        return
    c = I.lattice_config(a.config)
    dims = c["dims"]
    fat, lng = I.hisq_links(dims, c["seed"], c["eps"])
    ctx = H.hisq_create(dims, t_antiperiodic=True, device=0)
    H.hisq_load_links(ctx, fat, lng, long_recon=a.recon, long_scale=I.C3_NAIK if a.recon != 18 else 1.0)
    H.hisq_set_mass(ctx, c["mass"])
    if a.mrhs > 1:
        import numpy as np

        eta = np.stack([I.gaussian_source(dims, 11, j) for j in range(a.mrhs)])
    else:
        eta = I.gaussian_source(dims, 11, 0)
    prm = H.hisq_default_solve_params(tol=1e-14, max_iter=a.iters, precision_sloppy=a.sloppy,
                                      compute_full_residual=0, batch=1 if a.mrhs > 1 else 0,
                                      precision_reliable=a.reliable)
    _, st, status = H.hisq_solve(ctx, eta, prm)
    print(f"{a.config} {dims}: {st[0]['iterations']} iterations, status {status}")
    if a.tc > 0:
        import numpy as np

        from paper_2502_00152_gb300.inputs import random_normal

        V = I.volume(dims)
        par = (np.indices(dims[::-1]).sum(axis=0) & 1).reshape(-1)
        vecs = random_normal(5, 77, 0, 6 * V * a.tc).reshape(a.tc, V, 3, 2)
        vecs = vecs[..., 0] + 1j * vecs[..., 1]
        vecs[:, par == 1] = 0
        vecs /= np.linalg.norm(vecs.reshape(a.tc, -1), axis=1)[:, None, None]
        H.hisq_set_eigvecs(ctx, vecs, np.linspace(0.01, 0.1, a.tc), a.tc_prec)
        bs = np.stack([I.gaussian_field(dims, 40 + j) for j in range(24)])
        for _ in range(2):
            H.hisq_deflate_batch(ctx, bs)
        print(f"tensor-core deflation: {a.tc} vectors x 24 right-hand sides done")
    ctx.close()


if __name__ == "__main__":
    main()
