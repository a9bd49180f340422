"""Planted mistakes in the oracle are caught by its pins.

Each case copies ``oracle/sisu_oracle.c``, plants one plausible mistake (a
dropped term, a wrong sign, a wrong index, a transposed operand, a wrong
constant), compiles the copy on the CPU and runs the pin set: Python-integer
field checks, a FIPS 180 vector, the independent statement digest, the
brute-force prover and the verifier's accept/reject behaviour.  At least one
pin must fail for every mutant.
"""
import hashlib
import json
import os
import random
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth
from oracle import Oracle, brute
from oracle.binding import SRC, ints_to_bytes, bytes_to_ints

P = brute.P

MUTANTS = {
    "fold_sign": ("T[j * width + x] = fr_add(lo, fr_mul(r, fr_sub(hi, lo)));",
                  "T[j * width + x] = fr_add(lo, fr_mul(r, fr_sub(lo, hi)));"),
    "copy_line_sign": ("row[x] = fr_add(lo, fr_mul(tt, fr_sub(hi, lo)));",
                       "row[x] = fr_add(hi, fr_mul(tt, fr_sub(hi, lo)));"),
    "copy_drop_add_gates": ("/* entry e weighs w(out e) */\n                    S = fr_add(S,",
                            "/* entry e weighs w(out e) */\n                    if (cc->type[i][e]) S = fr_add(S,"),
    "eval_overwrites": ("out[cc->out[i][e]] = fr_add(out[cc->out[i][e]],", "out[cc->out[i][e]] = fr_add(fr_zero(),"),
    "eq1_dropped_term": ("return fr_add(fr_mul(a, b), fr_mul(fr_sub(one, a), fr_sub(one, b)));",
                         "return fr_add(fr_mul(a, b), fr_mul(fr_sub(one, a), b));"),
    "xphase_wrong_index": ("op_gate(ty, at, A0[cc->in2[i][q]])", "op_gate(ty, at, A0[cc->in1[i][q]])"),
    "yphase_transposed": ("op_gate(ty, vx, at)", "op_gate(ty, at, at)"),
    "omega_wrong_point": ("fr_mul(beta, eq_point_index(ry, cc->s[i], g)));\n        /* copy phase */",
                          "fr_mul(beta, eq_point_index(rx, cc->s[i], g)));\n        /* copy phase */"),
    "bit_order": ("return (int)((v >> (s - m)) & 1u);", "return (int)((v >> (m - 1)) & 1u);"),
    "barrett_quotient_word": ("q3[i] = q2[5 + i];", "q3[i] = q2[4 + i];"),
    "add_no_reduce": ("if (mw_cmp(s.w, MODW, 4) >= 0) mw_sub(s.w, s.w, MODW, 4);\n    return s;",
                      "if (mw_cmp(s.w, MODW, 4) > 0) mw_sub(s.w, s.w, MODW, 4);\n    return s;"),
    "sha_rotation": ("uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);",
                     "uint32_t S1 = rotr(e, 6) ^ rotr(e, 12) ^ rotr(e, 25);"),
    "challenge_mask": ("hm[31] &= 0x3f;", "hm[31] &= 0x1f;"),
    "merkle_tag": ("msg[64] = 0x01;", "msg[64] = 0x00;"),
    "verifier_skips_final": ("if (!fr_eq(claim, fr_mul(e, sum))) { ok = 0; break; }",
                             "if (0) { ok = 0; break; }"),
    "verifier_skips_input": ("if (!fr_eq(vy, mle_by_folding(Vin, c + s, pt))) { ok = 0; break; }",
                             "if (0) { ok = 0; break; }"),
    "verifier_g1_sign": ("g[0] = sent[0]; g[2] = sent[1]; g[3] = sent[2];\n            g[1] = fr_sub(claim, g[0]);",
                         "g[0] = sent[0]; g[2] = sent[1]; g[3] = sent[2];\n            g[1] = fr_sub(g[0], claim);"),
    "prover_sends_g1": ("sent[0] = g[0];\n    for (int t = 2; t < n; ++t) sent[t - 1] = g[t];",
                        "sent[0] = g[0];\n    for (int t = 2; t < n; ++t) sent[t - 1] = g[t - 1];"),
    "assoc_constant": ("const fr big = fr_u64(4294967295u);", "const fr big = fr_u64(4294967296u);"),
    "assoc_square": ("r = fr_mul(fr_mul(t, t), t);", "r = fr_mul(t, t);"),
    "assoc_no_chain": ("fr t = fr_add(fr_add(r, e), big);", "fr t = fr_add(e, big);"),
    "distinct_allows_equal": ("if (mw_cmp(cur.w, prev.w, 4) <= 0) return 0;", "if (mw_cmp(cur.w, prev.w, 4) < 0) return 0;"),
    "interp_wrong_node": ("num = fr_mul(num, fr_sub(x, fr_u64((uint64_t)j)));",
                          "num = fr_mul(num, fr_sub(x, fr_u64((uint64_t)j + 1)));"),
    # general circuits (Sec. 2.7)
    "general_block_base": ("        uint32_t u = gc->bbase[i][b] + k;\n        M[gc->bys[i][b][k]]",
                           "        uint32_t u = k;\n        M[gc->bys[i][b][k]]"),
    "general_first_term_only": ("for (uint32_t t = 0; t < terms[i].n; ++t) gcopy_round(",
                                "for (uint32_t t = 0; t < 1 && t < terms[i].n; ++t) gcopy_round("),
    "general_copy_weight_dropped": ("om[g] = fr_add(om[g], fr_mul(e, terms[i].M[t][g]));",
                                    "om[g] = fr_add(om[g], terms[i].M[t][g]);"),
    "general_used_index": ("if (gc->src[i][g] == j) gc->u2[i][g] = (uint32_t)pos[gc->in2[i][g]];",
                           "if (gc->src[i][g] == j) gc->u2[i][g] = base - cnt;"),
    "general_phase2_first_input": ("pre[g] = eq_point_index(rx, sx, gc->in1[i][g]);",
                                   "pre[g] = eq_point_index(rx, sx, gc->u2[i][g]);"),
    # the transcript: an absorb's count tweak cut to three bits (wrong only
    # for the long layer-end absorbs of general layers reading many layers)
    "absorb_count_low_bits": ("t->st[31] ^= (uint8_t)n;", "t->st[31] ^= (uint8_t)(n & 7);"),
    "general_block_values_swapped": ("vb[b] = fr_add(vb[b], fr_mul(eq_point_index(rx, sx, u), A0[u]));",
                                     "vb[b] = fr_add(vb[b], fr_mul(eq_point_index(ry, sx, u), A0[u]));"),
}


def _pins(o: Oracle) -> list:
    """Names of the pins that fail for this build of the oracle."""
    failed = []
    rng = random.Random(1)
    a = [rng.randrange(P) for _ in range(64)] + [P - 1, 0, 1]
    b = [rng.randrange(P) for _ in range(64)] + [P - 1, P - 1, P - 1]
    try:
        for op, fn in ((0, lambda x, y: (x + y) % P), (1, lambda x, y: (x - y) % P), (2, lambda x, y: x * y % P)):
            if bytes_to_ints(o.fr_op(op, ints_to_bytes(a), ints_to_bytes(b))) != [fn(x, y) for x, y in zip(a, b)]:
                failed.append(f"field{op}")
    except ValueError:
        failed.append("field-error")
    if o.sha256(b"abc") != hashlib.sha256(b"abc").digest():
        failed.append("sha")
    data = bytes(range(256)) * 13
    if o.statement_digest(data) != brute.digest(data):
        failed.append("digest")
    for C, widths, pct in ((4, [4, 4, 4], 50), (3, [3, 5, 2], 50), (2, [4, 2, 4], 100)):
        circ = synth.micro(5, C, widths, pct)
        x = synth.inputs_for(circ)
        xb = synth.fr_bytes(x)
        try:
            proof = o.prove(circ, xb)
        except ValueError:
            failed.append("prove-error")
            continue
        if proof != brute.prove(circ, synth.fr_ints(x)):
            failed.append(f"brute{C}")
        outs = brute.evaluate(brute.Padded(circ), synth.fr_ints(x))[0]
        outs_real = b"".join(brute.fe(outs[bb * brute.Padded(circ).W[0] + g])
                             for bb in range(C) for g in range(widths[0]))
        if o.verify(circ, xb, outs_real, proof) != 0:
            failed.append(f"accept{C}")
        honest = brute.prove(circ, synth.fr_ints(x))
        hdr = 8 + 4 * (circ.depth + 3)
        for k in range(0, (len(honest) - hdr) // 32):
            bad = bytearray(honest)
            bad[hdr + 32 * k] ^= 1
            if o.verify(circ, xb, outs_real, bytes(bad)) == 0:
                failed.append(f"reject{C}")
                break
        # an honest-looking proof over other inputs than the statement's
        fake = synth.fr_ints(x)
        fake[1] = (fake[1] + 1) % P
        forged = brute.prove(circ, fake, statement_inputs=synth.fr_ints(x))
        fake_outs = brute.evaluate(brute.Padded(circ), fake)[0]
        fake_real = b"".join(brute.fe(fake_outs[bb * brute.Padded(circ).W[0] + g])
                             for bb in range(C) for g in range(widths[0]))
        if o.verify(circ, xb, fake_real, forged) == 0:
            failed.append(f"forged-inputs{C}")
    # round-consistent proof of false outputs for a one-layer circuit
    circ = synth.micro(6, 4, [4, 4], 50)
    x = synth.fr_ints(synth.inputs_for(circ))
    outs = brute.evaluate(brute.Padded(circ), x)[0]
    outs[0] = (outs[0] + 1) % P
    forged = brute.forge_one_layer(circ, x, outs)
    if o.verify(circ, ints_to_bytes(x), ints_to_bytes(outs), forged) == 0:
        failed.append("forged-final")
    # consistent proof whose v_y is false at the input layer
    outs = brute.evaluate(brute.Padded(circ), x)[0]
    forged = brute.forge_vy_one_layer(circ, x)
    if o.verify(circ, ints_to_bytes(x), ints_to_bytes(outs), forged) == 0:
        failed.append("forged-vy")
    # accumulation gates (Sec. 3.4.3): several entries summed into a gate
    acc = synth.accumulation_circuit(7, 2, [3, 4, 4], 3)
    xa = synth.inputs_for(acc)
    try:
        if o.prove(acc, synth.fr_bytes(xa)) != brute.prove(acc, synth.fr_ints(xa)):
            failed.append("brute-acc")
    except ValueError:
        failed.append("prove-acc-error")
    # general circuits (Sec. 2.7): against the brute-force prover, accepted,
    # every tampered element rejected
    for seed, C, widths, far in ((5, 4, [8, 8, 6, 8], 40), (7, 2, [8, 4, 8, 4], 70), (31, 2, [4] * 7, 100)):
        gcirc = synth.general_circuit(seed, C, widths, 50, far)
        xg = synth.inputs_for(gcirc)
        xgb = synth.fr_bytes(xg)
        try:
            gp = o.prove_general(gcirc, xgb)
            gouts = o.outputs_general(gcirc, xgb)
        except ValueError:
            failed.append("prove-general-error")
            continue
        honest = brute.prove_general(gcirc, synth.fr_ints(xg))
        if gp != honest:
            failed.append(f"brute-general{seed}")
        pg = brute.GeneralPadded(gcirc)
        vg = brute.evaluate_general(pg, synth.fr_ints(xg))[0]
        real = b"".join(brute.fe(vg[bb * pg.W[0] + g]) for bb in range(C) for g in range(widths[0]))
        if o.verify_general(gcirc, xgb, real, honest) != 0:
            failed.append(f"accept-general{seed}")
        hdr = 8 + 4 * (gcirc.depth + 3)
        for k in range(0, (len(honest) - hdr) // 32, 3):
            bad = bytearray(honest)
            bad[hdr + 32 * k] ^= 1
            if o.verify_general(gcirc, xgb, real, bytes(bad)) == 0:
                failed.append(f"reject-general{seed}")
                break
    # associative hash (Sec. 3.4.1): closed forms at e + 2^32 - 1 = 1 and 2;
    # pairwise-distinct check (Sec. 3.4.2) on a list with a repeat
    try:
        got = bytes_to_ints(o.assoc_F(ints_to_bytes([(1 - (2**32 - 1)) % P, (2 - (2**32 - 1)) % P])))
        if got != [729, 1006012008]:
            failed.append("assoc-closed-form")
        if o.pairwise_distinct_check(ints_to_bytes([7, 3, 7]), ints_to_bytes([3, 7, 7])) != 0:
            failed.append("distinct-repeat")
        if o.pairwise_distinct_check(ints_to_bytes([7, 3, 9]), ints_to_bytes([3, 7, 9])) != 1:
            failed.append("distinct-accept")
    except ValueError:
        failed.append("assoc-error")
    return failed


def test_unmutated_oracle_passes_all_pins(oracle):
    assert _pins(oracle) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = str(tmp_path / f"libmutant_{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-w", "-shared", "-fPIC", "-o", lib, str(path)])
    # A mutant may loop for ever (a wrong Barrett quotient leaves a huge
    # remainder to subtract): run its pins in a child process with a limit.
    try:
        res = subprocess.run([sys.executable, os.path.abspath(__file__), lib], capture_output=True,
                             text=True, timeout=45)
        failed = json.loads(res.stdout.strip().splitlines()[-1]) if res.returncode == 0 else ["crash"]
    except subprocess.TimeoutExpired:
        failed = ["timeout"]
    assert failed, f"mutant {name} passed every pin"


if __name__ == "__main__":
    print(json.dumps(_pins(Oracle(sys.argv[1]))))
