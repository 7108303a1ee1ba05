"""Builds the CUDA library libsmc.so in-tree (paper_0912_2551_gb300/_build/)
with nvcc for sm_103a: the translation units compile in parallel, then link."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
BUILD = os.path.join(HERE, '_build')
LIB = os.path.join(BUILD, 'libsmc.so')
SOURCES = ['smc_kernels.cu', 'smc_api.cu', 'smc_compile.cpp', 'smc_mlp.cu', 'smc_jit.cpp', 'smc_cme.cu']
HEADERS = ['smc_internal.h', 'smc_compile.h', 'smc_nest.h', 'smc_mlp.h', 'smc_mlp_train.cuh', 'smc_tc.h', 'smc_device.cuh', 'smc_jit.h',
           'smc_jit_kernel.cuh', 'nvrtc_stdint.h', 'smc_cme.h', 'smc_fp64i.h']
# sources of the run-time compiled kernels, embedded into the library as
# (include name, file) pairs
JIT_EMBED = [('stdint.h', 'nvrtc_stdint.h'), ('smc_fp64i.h', 'smc_fp64i.h'), ('smc_internal.h', 'smc_internal.h'),
             ('smc_device.cuh', 'smc_device.cuh'), ('smc_jit_kernel.cuh', 'smc_jit_kernel.cuh')]
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']


def _nvcc():
    for c in (os.environ.get('NVCC'), '/usr/local/cuda/bin/nvcc', 'nvcc'):
        if c and (os.path.exists(c) or c == 'nvcc'):
            return c
    raise RuntimeError('nvcc not found')


def _inputs():
    srcs = [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    hdrs = [os.path.join(CSRC, h) for h in HEADERS if os.path.exists(os.path.join(CSRC, h))]
    hdrs.append(os.path.join(os.path.dirname(HERE), 'include', 'smc.h'))
    return srcs, hdrs


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    srcs, hdrs = _inputs()
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in srcs + hdrs + [__file__])


def _write_embedded_sources():
    """_build/smc_jit_sources.inc: the run-time compiled kernel's headers as
    C++ raw string literals."""
    names, bodies = [], []
    for name, fname in JIT_EMBED:
        with open(os.path.join(CSRC, fname)) as f:
            text = f.read()
        if ')SMCJIT"' in text:
            raise RuntimeError(f'{fname} contains the raw-string delimiter')
        names.append(name)
        bodies.append(text)
    out = ['// generated by build.py from csrc/: do not edit']
    out.append('static const char *const kJitHeaderNames[] = {' + ', '.join(f'"{n}"' for n in names) + '};')
    out.append('static const char *const kJitHeaderSources[] = {')
    out += [f'R"SMCJIT({b})SMCJIT",' for b in bodies]
    out.append('};')
    path = os.path.join(BUILD, 'smc_jit_sources.inc')
    text = '\n'.join(out) + '\n'
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, 'w') as f:
            f.write(text)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    _write_embedded_sources()
    nvcc = _nvcc()
    srcs, _ = _inputs()
    # host code: no contraction into fused multiply-adds, so the host's Eq. 4 /
    # Eq. 5 arithmetic rounds every operation as written on x86 and Arm alike
    common = ARCH + ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '-Xcompiler', '-O2',
                     '-Xcompiler', '-ffp-contract=off',
                     '-I', CSRC, '-I', BUILD, '-I', os.path.join(os.path.dirname(HERE), 'include')]
    if verbose:
        common += ['-Xptxas', '-v']

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + '.o')
        cmd = [nvcc] + common + ['-c', src, '-o', obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f'nvcc failed on {src}:\n{r.stdout}\n{r.stderr}')
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f'.{os.getpid()}.tmp'
    cmd = [nvcc] + ARCH + ['-shared', '-o', tmp] + objs + ['-lcudart_static', '-lrt', '-lpthread', '-ldl']
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f'link failed:\n{r.stdout}\n{r.stderr}')
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    print(build(force='--force' in sys.argv, verbose='-v' in sys.argv))
