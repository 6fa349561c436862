"""The build compiles every CUDA source of the library; sweep.cu as three objects (host
helpers, FP32 and FP64 kernel instantiations) and sweep_reg.cu as one object per
register-sweep kernel plus its dispatch table, so that the long compiles run in
parallel."""
import os

from paper_1609_07758_gb300 import build


def test_every_source_is_compiled_and_sweep_in_three_parts():
    jobs = build.jobs()
    srcs = build.sources()
    assert srcs and {j[0] for j in jobs} == set(srcs)
    names = [j[2] for j in jobs]
    assert len(names) == len(set(names))                      # distinct object files
    sweep = [j for j in jobs if os.path.basename(j[0]) == "sweep.cu"]
    assert sorted(j[1] for j in sweep) == [f"HOFEM_SWEEP_PART={k}" for k in range(3)]
    reg = [j for j in jobs if os.path.basename(j[0]) == "sweep_reg.cu"]
    assert sorted(j[1] for j in reg) == sorted([f"HOFEM_REG_PART={k}" for k in range(15)] + ["HOFEM_REG_PART=100"])
    assert all(j[1] is None for j in jobs if os.path.basename(j[0]) not in ("sweep.cu", "sweep_reg.cu"))
