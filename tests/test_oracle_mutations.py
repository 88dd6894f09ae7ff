"""Mutation check of the oracle's pins (CPU only).

Each mutant plants one plausible mistake in a copy of one oracle module (a dropped conjugate or
term, a wrong sign, a transposed index, a swapped axis, a sum for a mean, an off-by-one) and runs
that module's pins against the copy in a scratch directory; the pins must fail on every mutant,
by a failing assertion (not an import error). An unmutated copy run the same way must pass, so a
failure means the pins caught the planted mistake, not a broken harness. The real oracle is never
modified.

Only the parts that something outside the oracle fixes are mutated: the network's architecture
and the synthetic lattice's constants are this build's choices (no pin can fix them), its
gradients and sampling rules are not.
"""
import concurrent.futures as cf
import os
import pathlib
import shutil
import subprocess
import sys

ROOT = pathlib.Path(__file__).resolve().parents[1]

# (name, exact text occurring once in the module, replacement)
PC_ENGINE = [
    ("Eq. 7 axes swapped", "g = gy[:, None] * gx[None, :]", "g = gx[:, None] * gy[None, :]"),
    ("Eq. 7 kernel not normalised", "    return g / g.sum()", "    return g"),
    ("Fresnel phase sign", "np.exp(-1j * np.pi * (u[:, None] ** 2", "np.exp(1j * np.pi * (u[:, None] ** 2"),
    ("far field not centred", "return np.fft.fftshift(np.fft.fft2(psi), axes=(-2, -1))", "return np.fft.fft2(psi)"),
    ("back-propagation without conj(H)", "np.fft.fft2(Psi) * np.conj(H)", "np.fft.fft2(Psi) * H"),
    ("mode sum replaced by a maximum", "S = np.sum(np.abs(Psi) ** 2, axis=0)", "S = np.max(np.abs(Psi) ** 2, axis=0)"),
    ("Eq. 6 model not squared", "        Ihat = AG ** 2", "        Ihat = AG"),
    ("Eq. 2 ratio without sqrt(I)", "R = np.sqrt(I_n) / np.sqrt(Im + eps * eps)", "R = I_n / np.sqrt(Im + eps * eps)"),
    ("blur domains swapped", 'if blur_domain == "amplitude":', 'if blur_domain != "amplitude":'),
    ("Eq. 11 without absolute value", "num = np.sum(np.abs(lna[y:y + M, x:x + M]))", "num = np.sum(lna[y:y + M, x:x + M])"),
    ("per-pixel C as a sum, not a mean", "C = np.where(covered, csum / np.maximum(cnt, 1.0), 1.0)",
     "C = np.where(covered, csum, 1.0)"),
    ("Eq. 9 sign", "(1.0 - prm.alpha1) * lna + prm.alpha1 * C * phi", "(1.0 - prm.alpha1) * lna - prm.alpha1 * C * phi"),
    ("Eq. 10 C not inverted", "prm.alpha2 * lna / C", "prm.alpha2 * lna * C"),
    ("step without the delta term", "(c_den * den[reached] + c_max * den.max())", "(c_den * den[reached])"),
    ("object numerator without conj(P)",
     "        NO[y:y + M, x:x + M] += np.sum(np.conj(P) * dpsi, axis=0)\n        DO[y:y + M, x:x + M] += P2\n"
     "        NP += np.conj(o)[None] * dpsi",
     "        NO[y:y + M, x:x + M] += np.sum(P * dpsi, axis=0)\n        DO[y:y + M, x:x + M] += P2\n"
     "        NP += np.conj(o)[None] * dpsi"),
    ("probe numerator without conj(o)", "        NP += np.conj(o)[None] * dpsi", "        NP += o[None] * dpsi"),
    ("probe denominator |o| not squared", "        NP += np.conj(o)[None] * dpsi\n        DP += np.abs(o) ** 2",
     "        NP += np.conj(o)[None] * dpsi\n        DP += np.abs(o)"),
    ("object denominator from the first mode only", "    P2 = np.sum(np.abs(P) ** 2, axis=0)\n    errnum = []",
     "    P2 = np.abs(P[0]) ** 2\n    errnum = []"),
    ("box gathered transposed", "        o = O[y:y + M, x:x + M]\n        psi = P * o[None]",
     "        o = O[x:x + M, y:y + M]\n        psi = P * o[None]"),
    ("error denominator sum I, not sum I^2", "errden = [math.fsum((I[n].astype(np.float64) ** 2).ravel())",
     "errden = [math.fsum((I[n].astype(np.float64)).ravel())"),
    ("error not square-rooted", "    E = math.sqrt(math.fsum(errnum) / math.fsum(errden))",
     "    E = math.fsum(errnum) / math.fsum(errden)"),
    ("probe step starts one iteration late", "    if t >= prm.probe_update_start:\n        P_new = P + np.stack",
     "    if t > prm.probe_update_start:\n        P_new = P + np.stack"),
    ("pc-DM reflection 2 psi_ov - psi lost", "chi = 2.0 * psi_ov - psi[n]", "chi = psi_ov - psi[n]"),
    ("pc-DM state replaced, not differenced", "psi[n] = psi[n] + propagate_backward(Chi_new, prm) - psi_ov",
     "psi[n] = propagate_backward(Chi_new, prm)"),
    ("window excludes its first iteration", "return any(lo <= t <= hi for (lo, hi) in windows)",
     "return any(lo < t <= hi for (lo, hi) in windows)"),
    ("C_n not clamped", "out[n] = min(max(num / den, cmin), cmax)", "out[n] = num / den"),
    ("constraint touches uncovered pixels", "return np.where(covered, a_c * np.exp(1j * phi_c), O)",
     "return a_c * np.exp(1j * phi_c)"),
    ("Eq. 6 blurs the intensity, then takes the root", "AG = blur(np.sqrt(S), g)", "AG = np.sqrt(blur(S, g))"),
    ("modulus keeps |Psi| only", "return R[None] * Psi, Ihat", "return R[None] * np.abs(Psi), Ihat"),
    ("rPIE object denominator without (1 - alpha)", "return (1.0 - prm.rpie_alpha_obj, prm.rpie_alpha_obj),",
     "return (1.0, prm.rpie_alpha_obj),"),
    ("probe step with the object's beta",
     "        P_new = P + np.stack([_normalised_step(prm.beta_probe, NP[k], DP, *c_probe) for k in range(K)])\n"
     "    else:\n        P_new = P.copy()\n    return O_new, P_new, errnum",
     "        P_new = P + np.stack([_normalised_step(prm.beta_obj, NP[k], DP, *c_probe) for k in range(K)])\n"
     "    else:\n        P_new = P.copy()\n    return O_new, P_new, errnum"),
    ("batches all start from the iteration's state", "        O, P, en = _batch_step(I, positions, parts[b], O, P, prm, t, eps, g)",
     "        O1, P1, en = _batch_step(I, positions, parts[b], O if b < 0 else O, P, prm, t, eps, g)\n"
     "        O, P = (O1, P1) if b == len(parts) - 1 else (O, P)"),
    ("last batch dropped", "return [perm[b:b + prm.minibatch] for b in range(0, N, prm.minibatch)]",
     "return [perm[b:b + prm.minibatch] for b in range(0, N - prm.minibatch, prm.minibatch)]"),
]

MONO = [
    ("magnification inverted", "        t = c + (i - c) / a\n", "        t = c + (i - c) * a\n"),
    ("interpolation weights swapped", "            S[i, i0] += 1.0 - f", "            S[i, i0] += f"),
    ("line weight not divided by a^2", "float(w) / (float(a) * float(a))", "float(w) / float(a)"),
    ("adjoint with the forward's transposes", "sum(w * (S.T @ R @ S) for w, S in ops)",
     "sum(w * (S @ R @ S.T) for w, S in ops)"),
    ("CGLS step size", "        alpha = gamma / qq\n", "        alpha = gamma / math.sqrt(qq)\n"),
    ("CGLS residual sign", "        r = r - alpha * q\n", "        r = r + alpha * q\n"),
    ("CGLS direction ratio inverted", "p = s + (gamma_new / gamma) * p", "p = s + (gamma / gamma_new) * p"),
    ("clamp as an absolute value", "X = np.maximum(X, 0.0)", "X = np.abs(X)"),
]

UNET = [
    ("output gradient without the factor 2", "d_out = rd(2.0 * (out - target) / n_out)", "d_out = rd((out - target) / n_out)"),
    ("ReLU mask dropped", 'd_c2 = rd(d_a2 * (c["a2"] > 0))', "d_c2 = rd(d_a2)"),
    ("skip-connection gradient dropped", "d_a1 = avgpool2_backward(d_p1) + d_a1_skip", "d_a1 = avgpool2_backward(d_p1)"),
    ("pooling gradient scale", "np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0",
     "np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 2.0"),
    ("sigma gradient without lambda", "d_sigma = 2.0 * lam * (sigma - sigma_t) / len(sigma)",
     "d_sigma = 2.0 * (sigma - sigma_t) / len(sigma)"),
    ("global-pool gradient not averaged", "[:, None, None, :] / hw", "[:, None, None, :]"),
    ("data gradient with flipped taps", 'np.einsum("nijo,oc->nijc", dy, w[:, t, :])',
     'np.einsum("nijo,oc->nijc", dy, w[:, 8 - t, :])'),
    ("bias gradient over one image", "return dxp[:, 1:-1, 1:-1], dw, dy.sum(axis=(0, 1, 2))",
     "return dxp[:, 1:-1, 1:-1], dw, dy[0].sum(axis=(0, 1))"),
]

WARMSTART = [
    ("lattice not at 60 degrees",
     "a2 = a * np.array([math.cos(theta + math.pi / 3), math.sin(theta + math.pi / 3)])",
     "a2 = a * np.array([math.cos(theta + math.pi / 4), math.sin(theta + math.pi / 4)])"),
    ("vacancy test inverted", "present = words[:, 0] >= np.uint64(vacancy_threshold(vacancy))",
     "present = words[:, 0] < np.uint64(vacancy_threshold(vacancy))"),
    ("peak width", "np.exp(-d2 / (2.0 * s_pk * s_pk))", "np.exp(-d2 / (s_pk * s_pk))"),
    ("pattern blur taps not normalised", "    g = np.exp(-d ** 2 / (2.0 * sigma * sigma))\n    return g / g.sum()",
     "    g = np.exp(-d ** 2 / (2.0 * sigma * sigma))\n    return g"),
    ("dose not normalised", "return I * (dose / I.sum())", "return I * dose"),
    ("Hann window off by half a sample", "np.sin(np.pi * (np.arange(Q) + 0.5) / Q) ** 2", "np.sin(np.pi * np.arange(Q) / Q) ** 2"),
    ("stitch not divided by the window sum", "out[covered] = num[covered] / den[covered]", "out[covered] = num[covered]"),
    ("median of an even count", "0.5 * (v[n // 2 - 1] + v[n // 2])", "v[n // 2]"),
]

PHILOX = [
    ("nine rounds", "    for _ in range(10):", "    for _ in range(9):"),
    ("key words swapped in the round", "c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0",
     "c0, c1, c2, c3 = hi1 ^ c1 ^ k1, lo1, hi0 ^ c3 ^ k0, lo0"),
    ("Weyl increments swapped", "k0 = (k0 + np.uint64(_W0)) & np.uint64(_MASK)", "k0 = (k0 + np.uint64(_W1)) & np.uint64(_MASK)"),
    ("shuffle range off by one", "j = int((int(wi) * (int(ii) + 1)) >> 32)", "j = int((int(wi) * int(ii)) >> 32)"),
]

MODULES = {
    "pc_engine.py": (["test_oracle_pins.py"], PC_ENGINE),
    "mono.py": (["test_oracle_mono.py"], MONO),
    "unet.py": (["test_oracle_unet.py"], UNET),
    "warmstart.py": (["test_oracle_warmstart.py"], WARMSTART),
    "philox.py": (["test_oracle_warmstart.py", "test_oracle_pins.py"], PHILOX),
}


def _scratch(tmp: pathlib.Path, module, mutant):
    """A copy of what the pins import (oracle, synth, the pin files, their conftest and golden
    files), with the mutant applied to the copy of oracle/<module>."""
    shutil.copytree(ROOT / "oracle", tmp / "oracle", ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(ROOT / "synth", tmp / "synth", ignore=shutil.ignore_patterns("__pycache__"))
    (tmp / "tests").mkdir()
    for f in ["conftest.py"] + sorted({p for pins, _ in MODULES.values() for p in pins}):
        shutil.copy(ROOT / "tests" / f, tmp / "tests" / f)
    shutil.copytree(ROOT / "tests" / "golden", tmp / "tests" / "golden")
    if mutant is not None:
        _, old, new = mutant
        path = tmp / "oracle" / module
        src = path.read_text()
        assert src.count(old) == 1, f"{module}: mutant site not unique or missing: {old!r}"
        path.write_text(src.replace(old, new))


def _run_pins(job) -> int:
    tmp, pins = job
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    env.pop("PYTHONPATH", None)
    r = subprocess.run([sys.executable, "-m", "pytest", *[f"tests/{p}" for p in pins], "-x", "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=tmp, env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, timeout=600)
    return r.returncode


def test_every_planted_mistake_fails_a_pin(tmp_path):
    all_pins = sorted({p for pins, _ in MODULES.values() for p in pins})
    jobs, names = [], []
    d = tmp_path / "control"
    d.mkdir()
    _scratch(d, None, None)
    jobs.append((d, all_pins))
    for module, (pins, mutants) in MODULES.items():
        for i, m in enumerate(mutants):
            d = tmp_path / f"{module[:-3]}_{i}"
            d.mkdir()
            _scratch(d, module, m)
            jobs.append((d, pins))
            names.append(f"{module}: {m[0]}")
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        rcs = list(ex.map(_run_pins, jobs))
    assert rcs[0] == 0, "the unmutated copy must pass its pins (harness check)"
    survivors = [n for n, rc in zip(names, rcs[1:]) if rc == 0]
    assert not survivors, f"mutants not caught by any pin: {survivors}"
    # caught by a failing pin (pytest exit code 1), not by an import or collection error
    broken = [(n, rc) for n, rc in zip(names, rcs[1:]) if rc != 1]
    assert not broken, f"mutants that did not run the pins: {broken}"
