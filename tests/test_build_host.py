"""The in-tree build's translation units (host only, nothing is compiled):
every source under csrc/ is built, the kernel instantiation sources once per
tile width with that width's define, and no two units share an object."""
import os

from paper_2301_03598_gb300 import build


def test_every_source_is_a_unit():
    srcs = {os.path.basename(s) for s in build.sources()}
    built = {os.path.basename(src) for src, _, _ in build.units()}
    assert srcs == built
    assert {"capi.cu", "planner.cpp", "kernels_bn.cu", "kernels_f8.cu"} <= srcs


def test_kernel_sources_compile_once_per_tile_width():
    defs = {}
    for src, obj, flags in build.units():
        defs.setdefault(os.path.basename(src), []).append(tuple(flags))
    assert sorted(defs["kernels_bn.cu"]) == [("-DSK_BN=128",), ("-DSK_BN=256",), ("-DSK_BN=64",)]
    assert sorted(defs["kernels_f8.cu"]) == [("-DSK_F8_BN=128",), ("-DSK_F8_BN=256",)]
    for name, variants in defs.items():
        if name not in ("kernels_bn.cu", "kernels_f8.cu"):
            assert variants == [()]


def test_objects_are_distinct_and_in_the_build_folder():
    objs = [obj for _, obj, _ in build.units()]
    assert len(objs) == len(set(objs))
    assert all(os.path.dirname(o) == build.OUT_DIR and o.endswith(".o") for o in objs)


def test_one_gencode_for_sm_103a():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
