"""Plausible mistakes to plant in the oracle (`oracle/edac_oracle.c`), one per entry: each is a
list of (text, replacement) pairs, every text occurring exactly once in the source.  Every
mistake but the ones in EQUIVALENT must make at least one pin of `test_oracle_pins.py` fail
(`test_oracle_mutations.py` checks it, on request).  The names say what is wrong."""

MUTATIONS = {
    # ---- kernel, pass A and neighbour search
    'w_coef15': [
        ('    if (q <= 1.0) return pow5(3.0 - q) - 6.0 * pow5(2.0 - q) + 15.0 * pow5(1.0 - q);',
         '    if (q <= 1.0) return pow5(3.0 - q) - 6.0 * pow5(2.0 - q) + 16.0 * pow5(1.0 - q);'),
    ],
    'dw_mid': [
        ('    if (q <= 2.0) return -5.0 * (pow4(3.0 - q) - 6.0 * pow4(2.0 - q));',
         '    if (q <= 2.0) return -5.0 * (pow4(3.0 - q) - 5.0 * pow4(2.0 - q));'),
    ],
    'alpha2': [
        ('7.0 / (478.0 * M_PI * h * h)',
         '7.0 / (487.0 * M_PI * h * h)'),
    ],
    'rho_own_mass': [
        ('            rho += S->m[j] * w;',
         '            rho += S->m[i] * w;'),
    ],
    'vol_m_over_rho': [
        ('        S->V[i] = 1.0 / sw;',
         '        S->V[i] = S->m[i] / rho;'),
    ],
    'nnb_no_self': [
        ('        S->nnb[i] = L->start[i + 1] - L->start[i];',
         '        S->nnb[i] = L->start[i + 1] - L->start[i] - 1;'),
    ],
    'min_image_L': [
        ('        if (d > 0.5 * L) d -= L;\n        else if (d < -0.5 * L) d += L;',
         '        if (d > L) d -= L;\n        else if (d < -L) d += L;'),
    ],
    'bins_2x3': [
        ('        for (int ox = -1; ox <= 1; ox++) {\n            int bx = cx + ox;',
         '        for (int ox = 0; ox <= 1; ox++) {\n            int bx = cx + ox;'),
    ],
    # ---- walls
    'wall_noslip_sign': [
        ('else { ug = 2.0 * P->wall_u[wi] - uf; vg = 2.0 * P->wall_v[wi] - vf; }',
         'else { ug = 2.0 * P->wall_u[wi] + uf; vg = 2.0 * P->wall_v[wi] + vf; }'),
    ],
    'wall_slip_v': [
        ('if (P->wall_slip[wi]) { ug = uf; vg = -vf; }',
         'if (P->wall_slip[wi]) { ug = uf; vg = vf; }'),
    ],
    'wall_p_plain_mean': [
        ('                pw = sp / sw;',
         '                pw = mp / (double)nf;'),
    ],
    'wall_no_fluid_u': [
        ('            ug = P->wall_u[wi];\n            vg = P->wall_v[wi];',
         '            ug = 0.0;\n            vg = 0.0;'),
    ],
    'wall_ut_zero': [
        ('        S->ut[i] = ug;\n        S->vt[i] = vg;',
         '        S->ut[i] = 0.0;\n        S->vt[i] = 0.0;'),
    ],
    # ---- inlet mirror (Sec. 3.2) and inlet velocity
    'mirror_no_gradient': [
        ('        S->p[o] = pk + (double)P->mirror_sign * (rx * g[0] + ry * g[1]);',
         '        S->p[o] = pk;'),
    ],
    'mirror_point_shift': [
        ('            qx[nq] = 2.0 * P->x_in - S->x[i];',
         '            qx[nq] = 2.0 * P->x_in - S->x[i] + P->dx;'),
    ],
    'mirror_unit_volume': [
        ('        double Vl = S->m[l] / S->rho[l];',
         '        double Vl = 1.0;'),
    ],
    'mirror_xy_swapped': [
        ('            M[a][1] += xlk * row[a];\n            M[a][2] += ylk * row[a];',
         '            M[a][1] += ylk * row[a];\n            M[a][2] += xlk * row[a];'),
    ],
    'mirror_sep_sign': [
        ('        double r = sqrt(sep(P, S->x[l], S->y[l], xk, yk, &xlk, &ylk));',
         '        double r = sqrt(sep(P, xk, yk, S->x[l], S->y[l], &xlk, &ylk));'),
    ],
    'singular_fallback_zero': [
        ('            fk[f] = b[f][0] / M[0][0];\n            continue;',
         '            fk[f] = 0.0;\n            continue;'),
    ],
    'mirror_no_fluid_one': [
        ('        for (int f = 0; f < nf; f++) fk[f] = 0.0;\n        return 0;',
         '        for (int f = 0; f < nf; f++) fk[f] = 1.0;\n        return 0;'),
    ],
    'modes_k': [
        ('sin((double)(k + 1) * M_PI * (y - P->inlet_y0) / P->inlet_h)',
         'sin((double)(k + 2) * M_PI * (y - P->inlet_y0) / P->inlet_h)'),
    ],
    'modes_y0': [
        ('sin((double)(k + 1) * M_PI * (y - P->inlet_y0) / P->inlet_h)',
         'sin((double)(k + 1) * M_PI * (y) / P->inlet_h)'),
    ],
    'pulse_cos6': [
        ('cos(M_PI * (y - P->inlet_y0) / 12.0)',
         'cos(M_PI * (y - P->inlet_y0) / 6.0)'),
    ],
    'pulse_centre_t1': [
        ('exp(-(t - q[1]) * (t - q[1]) / q[3])',
         'exp(-(t - q[2]) * (t - q[2]) / q[3])'),
    ],
    'vortex_v_sign': [
        ('        *v = -q[0] * xr / den;',
         '        *v = q[0] * xr / den;'),
    ],
    'vortex_core2': [
        ('        double den = xr * xr + yr * yr + q[1];',
         '        double den = xr * xr + yr * yr + 2.0 * q[1];'),
    ],
    'ramp_no_clamp': [
        ('        *u = P->U * (t < q[0] ? t / q[0] : 1.0);',
         '        *u = P->U * t / q[0];'),
    ],
    # ---- pass B
    'ptil_weights_swapped': [
        ('double ptil = (rhoj * (S->p[i] - pavg) + rhoi * (S->p[j] - pavg)) / (rhoi + rhoj);',
         'double ptil = (rhoi * (S->p[i] - pavg) + rhoj * (S->p[j] - pavg)) / (rhoi + rhoj);'),
    ],
    'pavg_zero': [
        ('            pavg = sp / (double)S->nnb[i];',
         '            pavg = 0.0 * sp;'),
    ],
    'pavg_count_plus_one': [
        ('            pavg = sp / (double)S->nnb[i];',
         '            pavg = sp / (double)(S->nnb[i] + 1);'),
    ],
    'pavg_fluid_only': [
        ('            for (int t = L->start[i]; t < L->start[i + 1]; t++) sp += S->p[L->idx[t]];',
         '            for (int t = L->start[i]; t < L->start[i + 1]; t++)\n                if (S->tag[L->idx[t]] == ORC_FLUID) sp += S->p[L->idx[t]];'),
    ],
    'cij_product': [
        ('            double cij = Vi * Vi + Vj * Vj;',
         '            double cij = 2.0 * Vi * Vj;'),
    ],
    'visc_arith_mean': [
        ('double etil = etai + etaj > 0.0 ? 2.0 * etai * etaj / (etai + etaj) : 0.0;',
         'double etil = 0.5 * (etai + etaj);'),
    ],
    'visc_sign': [
        ('            double visc = etil * gdotr / (r2 + eh2);',
         '            double visc = -etil * gdotr / (r2 + eh2);'),
    ],
    'visc_no_reg': [
        ('            double visc = etil * gdotr / (r2 + eh2);',
         '            double visc = etil * gdotr / (r2 + 1e-300);'),
    ],
    'visc_kinematic': [
        ('            double etai = rhoi * P->nu, etaj = rhoj * P->nu;',
         '            double etai = P->nu, etaj = P->nu;'),
    ],
    'div_sign': [
        ('            sp_rate += (S->m[j] * rhoi / rhoj) * c2 * (uij * gx + vij * gy)',
         '            sp_rate -= (S->m[j] * rhoi / rhoj) * c2 * (uij * gx + vij * gy)'),
    ],
    'div_no_density_ratio': [
        ('            sp_rate += (S->m[j] * rhoi / rhoj) * c2 * (uij * gx + vij * gy)',
         '            sp_rate += (S->m[j]) * c2 * (uij * gx + vij * gy)'),
    ],
    'pdiff_sign': [
        ('+ (cij / mi) * etile * (S->p[i] - S->p[j]) * gdotr / (r2 + eh2);',
         '+ (cij / mi) * etile * (S->p[j] - S->p[i]) * gdotr / (r2 + eh2);'),
    ],
    'nu_edac_4': [
        ('    const double nu_edac = P->alpha * h * P->cs / 8.0;',
         '    const double nu_edac = P->alpha * h * P->cs / 4.0;'),
    ],
    'edac_kinematic': [
        ('            double ei = rhoi * nu_edac, ej = rhoj * nu_edac;',
         '            double ei = nu_edac, ej = nu_edac;'),
    ],
    'ap_diff_mi': [
        ('            + (cij / mi) * etile * (S->p[i] - S->p[j]) * gdotr / (r2 + eh2);',
         '            + (cij) * etile * (S->p[i] - S->p[j]) * gdotr / (r2 + eh2);'),
    ],
    'abg_sign': [
        ('            S->abu[i] = -P->pb / mi * bx;\n            S->abv[i] = -P->pb / mi * by;',
         '            S->abu[i] = P->pb / mi * bx;\n            S->abv[i] = P->pb / mi * by;'),
    ],
    'abg_without_cij': [
        ('            bx += cij * gx;\n            by += cij * gy;',
         '            bx += gx;\n            by += gy;'),
    ],
    'gravity_dropped': [
        ('            S->au[i] = sx / mi + P->gx;\n            S->av[i] = sy / mi + P->gy;',
         '            S->au[i] = sx / mi;\n            S->av[i] = sy / mi;'),
    ],
    'A_sign': [
        ('0.5 * (Aix + Ajx)',
         '-0.5 * (Aix + Ajx)'),
        ('0.5 * (Aiy + Ajy)',
         '-0.5 * (Aiy + Ajy)'),
    ],
    'A_transposed': [
        ('            double Aix = Ai * S->u[i], Aiy = Ai * S->v[i];\n            double Ajx = Aj * S->u[j], Ajy = Aj * S->v[j];',
         '            double ui_g = S->u[i] * gx + S->v[i] * gy, uj_g = S->u[j] * gx + S->v[j] * gy;\n            double Aix = Ai_f * (S->ut[i] - S->u[i]) * ui_g, Aiy = Ai_f * (S->vt[i] - S->v[i]) * ui_g;\n            double Ajx = rhoj * (S->ut[j] - S->u[j]) * uj_g, Ajy = rhoj * (S->vt[j] - S->v[j]) * uj_g;\n            (void)Ai; (void)Aj;'),
    ],
    'A_without_rho_i': [
        ('        double Ai_f = rhoi; /* A_i.gW = rho_i u_i ((u~_i - u_i) . gW) */',
         '        double Ai_f = 1.0;'),
    ],
    'A_without_rho_j': [
        ('            double Aj = rhoj * ((S->ut[j] - S->u[j]) * gx + (S->vt[j] - S->v[j]) * gy);',
         '            double Aj = ((S->ut[j] - S->u[j]) * gx + (S->vt[j] - S->v[j]) * gy);'),
    ],
    'grad_sign': [
        ('                gx = dw * dxs / r;\n                gy = dw * dys / r;\n            }\n            double rhoj',
         '                gx = -dw * dxs / r;\n                gy = -dw * dys / r;\n            }\n            double rhoj'),
    ],
    'uij_ghost_for_solid': [
        ('            double uij = S->u[i] - S->u[j], vij = S->v[i] - S->v[j];',
         '            double uij = S->ut[i] - S->u[j], vij = S->vt[i] - S->v[j];'),
    ],
    'rates_for_outlet': [
        ('        int do_fluid = (ti == ORC_FLUID || ti == ORC_INLET);',
         '        int do_fluid = (ti == ORC_FLUID || ti == ORC_INLET || ti == ORC_OUTLET);'),
    ],
    'no_rates_for_inlet': [
        ('        int do_fluid = (ti == ORC_FLUID || ti == ORC_INLET);',
         '        int do_fluid = (ti == ORC_FLUID);'),
    ],
    # ---- solid force (Eq. tvf-momentum_solid)
    'solid_no_visc': [
        ('                sx += cij * (-ptil * gx + visc * uij);\n                sy += cij * (-ptil * gy + visc * vij);',
         '                sx += cij * (-ptil * gx);\n                sy += cij * (-ptil * gy);'),
    ],
    'solid_ptil_pavg': [
        ('        if (P->use_pavg && (!do_solid || literal)) {',
         '        if (P->use_pavg) {'),
    ],
    'solid_force_sign': [
        ('        if (do_solid) {\n            S->fx[i] = sx;\n            S->fy[i] = sy;',
         '        if (do_solid) {\n            S->fx[i] = -sx;\n            S->fy[i] = -sy;'),
    ],
    'literal_fluid_only': [
        ('            if (do_solid && !literal && S->tag[j] != ORC_FLUID) continue;',
         '            if (do_solid && S->tag[j] != ORC_FLUID) continue;'),
    ],
    'literal_no_pavg': [
        ('        if (P->use_pavg && (!do_solid || literal)) {',
         '        if (P->use_pavg && !do_solid) {'),
    ],
    'drag_fy_from_fx': [
        ('                H.fy += S->fy[i];',
         '                H.fy += S->fx[i];'),
    ],
    'drag_all_walls': [
        ('            if (is_wall(t) && P->wall_drag[wall_index(t)]) {\n                H.fx',
         '            if (is_wall(t)) {\n                H.fx'),
    ],
    # ---- outlets (Secs. 3.1-3.4)
    'J2_sign': [
        ('        S->J2[i] = rc * (S->u[i] - S->ubar[i]) + (S->p[i] - S->pbar[i]);',
         '        S->J2[i] = rc * (S->u[i] - S->ubar[i]) - (S->p[i] - S->pbar[i]);'),
    ],
    'J2_no_rc': [
        ('        S->J2[i] = rc * (S->u[i] - S->ubar[i]) + (S->p[i] - S->pbar[i]);',
         '        S->J2[i] = (S->u[i] - S->ubar[i]) + (S->p[i] - S->pbar[i]);'),
    ],
    'J2_rc_rho': [
        ('    const double rc = P->rho0 * P->cs;\n#pragma omp parallel for schedule(static)\n    for (int i = 0; i < S->n; i++) {\n        if (S->tag[i] != ORC_FLUID) continue;',
         '    const double rc = P->cs;\n#pragma omp parallel for schedule(static)\n    for (int i = 0; i < S->n; i++) {\n        if (S->tag[i] != ORC_FLUID) continue;'),
    ],
    'acou_full_J2': [
        ('        double pa = 0.5 * J2, ua = J2 / (2.0 * rc);',
         '        double pa = J2, ua = J2 / rc;'),
    ],
    'acou_rc_rho': [
        ('    const double h = h_of(P);\n    const double rc = P->rho0 * P->cs;\n    int n = S->n;',
         '    const double h = h_of(P);\n    const double rc = P->cs;\n    int n = S->n;'),
    ],
    'intensity_rho_c': [
        ('        double inten = S->p[i] * S->p[i] / (2.0 * P->rho0 * P->cs);',
         '        double inten = S->p[i] * S->p[i] / (P->rho0 * P->cs);'),
    ],
    'I_thr_rho': [
        ('    return q * q / (2.0 * P->rho0 * P->cs);\n}',
         '    return q * q / (2.0 * P->cs);\n}'),
    ],
    'gate_strict': [
        ('        if (inten <= I) {',
         '        if (inten < 0.5 * I) {'),
    ],
    'gate_updates_index_anyway': [
        ('            rg[3 * k + 2] = S->p[i];\n            S->rpos[i] = (k + 1) % P->n_avg;\n        }',
         '            rg[3 * k + 2] = S->p[i];\n        }\n        S->rpos[i] = (S->rpos[i] + 1) % P->n_avg;'),
    ],
    'window2': [
        ('        for (int k = 0; k < P->n_avg; k++) {\n            su += rg',
         '        for (int k = 0; k < 2; k++) {\n            su += rg'),
        ('S->ubar[i] = su / (double)P->n_avg;',
         'S->ubar[i] = su / 2.0;'),
        ('S->vbar[i] = sv / (double)P->n_avg;',
         'S->vbar[i] = sv / 2.0;'),
        ('S->pbar[i] = sp / (double)P->n_avg;',
         'S->pbar[i] = sp / 2.0;'),
    ],
    'ring_fill_rpos': [
        ('    S->rpos[i] = 0;\n    S->ubar[i] = S->u[i];',
         '    S->rpos[i] = 1;\n    S->ubar[i] = S->u[i];'),
    ],
    'blue_zero': [
        ('(mr > 0 ? sjp / (double)mr : 0.0)',
         '(mr > 0 ? 0.0 * sjp : 0.0)'),
    ],
    'blue_J2_excludes_self': [
        ('            } else if (S->tag[j] == ORC_OUTLET && S->redp[j]) {',
         '            } else if (S->tag[j] == ORC_OUTLET && S->redp[j] && j != o) {'),
    ],
    'outlet_v_kept': [
        ('        S->v[o] = S->vbar[o];\n        S->p[o] = p;',
         '        S->p[o] = p;'),
    ],
    'shepard_unweighted': [
        ('        double shep = red ? (sw > 0.0 ? sf / sw : sfm / (double)nf) : 0.0;',
         '        double shep = red ? sfm / (double)nf : 0.0;'),
    ],
    'moc_ref_dropped': [
        ('            u = P->moc_u_ref + ua;\n            p = P->moc_p_ref + pa;',
         '            u = ua;\n            p = pa;'),
    ],
    'moc_J2_p_sign': [
        ('S->J2[i] = rc * (S->u[i] - P->moc_u_ref) + (S->p[i] - P->moc_p_ref);',
         'S->J2[i] = rc * (S->u[i] - P->moc_u_ref) - (S->p[i] - P->moc_p_ref);'),
    ],
    'mod_dn_adv_fluid_J2': [
        ('                double fj = kind == ORC_OUT_MOD_DONOTHING ? S->u[j] : S->J2[j];',
         '                double fj = S->J2[j];'),
    ],
    'mod_dn_blue_no_mean': [
        ('            advn[o] = red ? shep : (mr > 0 ? blue_adv : S->ubar[o]);',
         '            advn[o] = red ? shep : S->ubar[o];'),
    ],
    'char_blue_adv_ubar': [
        ('            adv = red ? u : (mr > 0 ? blue_adv : u);',
         '            adv = red ? u : (mr > 0 ? blue_adv : S->ubar[o]);'),
    ],
    'mirror_outlet_adv_U': [
        ('        S->advp[o] = S->u[o];\n        S->J2p[o] = 0.0;',
         '        S->advp[o] = P->U;\n        S->J2p[o] = 0.0;'),
    ],
    'outlet_mirror_keeps_red': [
        ('        S->J2p[o] = 0.0;\n        S->redp[o] = 0;\n    }\n    nlist_free(&L);\n    free(fo);',
         '        S->J2p[o] = 0.0;\n    }\n    nlist_free(&L);\n    free(fo);'),
    ],
    'outlet_values_before_reads': [
        ('    for (int t = 0; t < nq; t++) { /* written after all reads (the fields are inputs above) */',
         '    for (int t = 0; t < 0; t++) { /* written after all reads (the fields are inputs above) */'),
    ],
    'donothing_updates': [
        ('    if (kind == ORC_OUT_DONOTHING) return;',
         '    if (kind == ORC_OUT_DONOTHING + 100) return;'),
    ],
    # ---- recycling (end of Sec. 3.4)
    'spawn_offset': [
        ('        nx_[k] = S->x[i] - L_in;',
         '        nx_[k] = S->x[i] - L_in + P->dx;'),
    ],
    'spawn_keeps_p0': [
        ('        np_[k] = S->p[i];',
         '        np_[k] = 0.0;'),
    ],
    'delete_at_xout': [
        ('if (P->has_outlet && t == ORC_OUTLET && S->x[i] >= P->x_out + L_out) {',
         'if (P->has_outlet && t == ORC_OUTLET && S->x[i] >= P->x_out + L_out - P->dx) {'),
    ],
    'hybrid_cross_keeps_u': [
        ('            if (P->outlet_kind == ORC_OUT_HYBRID) {\n                S->u[i] = S->ubar[i];',
         '            if (0) {\n                S->u[i] = S->ubar[i];'),
    ],
    'cross_advp_u': [
        ('            S->advp[i] = S->ubar[i];\n            mflux += S->m[i];',
         '            S->advp[i] = S->u[i] + 0.01;\n            mflux += S->m[i];'),
    ],
    'mass_flux_no_dt': [
        ('    H->mass_flux = mflux / P->dt;',
         '    H->mass_flux = mflux;'),
    ],
    'mass_flux_counts_spawns': [
        ('            spawn[nspawn].id = S->id[i];',
         '            mflux += S->m[i];\n            spawn[nspawn].id = S->id[i];'),
    ],
    'no_ring_fill_on_spawn': [
        ('            ring_fill(P, S, i);\n            spawn[nspawn].id',
         '            spawn[nspawn].id'),
    ],
    'to_outlet_late': [
        ('} else if (P->has_outlet && t == ORC_FLUID && S->x[i] >= P->x_out) {',
         '} else if (P->has_outlet && t == ORC_FLUID && S->x[i] >= P->x_out + 0.5 * P->dx) {'),
    ],
    'inlet_to_fluid_late': [
        ('} else if (P->has_inlet && t == ORC_INLET && S->x[i] >= P->x_in) {',
         '} else if (P->has_inlet && t == ORC_INLET && S->x[i] >= P->x_in + 0.5 * P->dx) {'),
    ],
    'spawn_ids_reversed': [
        ('    qsort(spawn, (size_t)nspawn, sizeof(id_index), by_id);',
         ''),
    ],
    'new_id_gap': [
        ('        S->id[i] = S->next_id++;',
         '        S->id[i] = ++S->next_id;'),
    ],
    'init_next_id': [
        ('        if (S->id[i] >= S->next_id) S->next_id = S->id[i] + 1;',
         '        if (S->id[i] >= S->next_id) S->next_id = S->id[i] + 2;'),
    ],
    # ---- integrator and time
    'forward_euler': [
        ('        stage(P, S, 0.5 * P->dt);\n        if (orc_evaluate(P, S)) return S->error;\n',
         '        stage(P, S, 0.5 * P->dt);\n'),
    ],
    'pred_full_dt': [
        ('        stage(P, S, 0.5 * P->dt);\n',
         '        stage(P, S, P->dt);\n'),
    ],
    'x_with_midpoint_u': [
        ('            S->x[i] = wrap(S->x0[i] + tau * S->ut[i]',
         '            S->x[i] = wrap(S->x0[i] + tau * (S->u0[i] + 0.5 * tau * S->au[i])'),
    ],
    'ut_without_bg': [
        ('            S->ut[i] = S->u[i] + tau * S->abu[i];',
         '            S->ut[i] = S->u[i];'),
    ],
    'x_with_u': [
        ('            S->x[i] = wrap(S->x0[i] + tau * S->ut[i]',
         '            S->x[i] = wrap(S->x0[i] + tau * S->u[i]'),
    ],
    'outlet_moves_with_u': [
        ('            S->x[i] = S->x0[i] + tau * S->advp[i];',
         '            S->x[i] = S->x0[i] + tau * S->u[i];'),
    ],
    'inlet_velocity_at_tn': [
        ('            inlet_velocity(P, S->y0[i], S->t + tau, &uin, &vin);',
         '            inlet_velocity(P, S->y0[i], S->t, &uin, &vin);'),
    ],
    'stage_p_from_current': [
        ('            S->p[i] = S->p0[i] + tau * S->ap[i];',
         '            S->p[i] = S->p[i] + tau * S->ap[i];'),
    ],
    'stage_v_from_current': [
        ('            S->v[i] = S->v0[i] + tau * S->av[i];',
         '            S->v[i] = S->v[i] + tau * S->av[i];'),
    ],
    'inlet_stage_y_moves': [
        ('            S->x[i] = S->x0[i] + tau * uin;\n',
         '            S->x[i] = S->x0[i] + tau * uin;\n            S->y[i] = S->y0[i] + tau * vin + tau * 0.1;\n'),
    ],
    'inlet_ut_zero': [
        ('            S->ut[i] = uin;\n            S->vt[i] = vin;\n            S->x[i] = S->x0[i] + tau * uin;',
         '            S->ut[i] = 0.0;\n            S->vt[i] = vin;\n            S->x[i] = S->x0[i] + tau * uin;'),
    ],
    'init_ut_zero': [
        ('        S->ut[i] = S->u[i];\n        S->vt[i] = S->v[i];\n        ring_fill(P, S, i);',
         '        S->ut[i] = 0.0;\n        S->vt[i] = S->v[i];\n        ring_fill(P, S, i);'),
    ],
    'time_not_advanced': [
        ('        S->t = (double)S->nstep * P->dt;',
         '        S->t = (double)(S->nstep - 1) * P->dt;'),
    ],
    # ---- which tags take part, gate threshold, time levels, ill-conditioned mirror
    'inlet_mirror_all_tags': [
        ('            qy[nq] = S->y[i];\n            nq++;\n        }\n    nlist L;\n    build_lists(P, S, nq, qx, qy, 1u << ORC_FLUID, &L);\n#pragma omp parallel for schedule(static)\n    for (int t = 0; t < nq; t++) {\n        int o = who[t];\n        double pk',
         '            qy[nq] = S->y[i];\n            nq++;\n        }\n    nlist L;\n    build_lists(P, S, nq, qx, qy, 0xFFu, &L);\n#pragma omp parallel for schedule(static)\n    for (int t = 0; t < nq; t++) {\n        int o = who[t];\n        double pk'),
    ],
    'walls_see_inlet': [
        ('        for (int t = L->start[i]; t < L->start[i + 1]; t++) {\n            int j = L->idx[t];\n            if (S->tag[j] != ORC_FLUID) continue;\n            double r = sqrt(sep(P, S->x[i], S->y[i], S->x[j], S->y[j], &dx, &dy));\n            double w = orc_W(r, h);\n            sw += w;\n            sp += S->p[j] * w;',
         '        for (int t = L->start[i]; t < L->start[i + 1]; t++) {\n            int j = L->idx[t];\n            if (S->tag[j] != ORC_FLUID && S->tag[j] != ORC_OUTLET) continue;\n            double r = sqrt(sep(P, S->x[i], S->y[i], S->x[j], S->y[j], &dx, &dy));\n            double w = orc_W(r, h);\n            sw += w;\n            sp += S->p[j] * w;'),
    ],
    'red_by_inlet_too': [
        ('            if (S->tag[j] == ORC_FLUID) {\n                double r = sqrt(sep(P, S->x[o], S->y[o], S->x[j], S->y[j], &dx, &dy));',
         '            if (S->tag[j] == ORC_FLUID || S->tag[j] == ORC_WALL) {\n                double r = sqrt(sep(P, S->x[o], S->y[o], S->x[j], S->y[j], &dx, &dy));'),
    ],
    'i_thresh_zero_ignored': [
        ('    if (P->i_thresh >= 0.0) return P->i_thresh;',
         '    if (P->i_thresh > 0.0) return P->i_thresh;'),
    ],
    'ring_for_outlet_too': [
        ('        if (S->tag[i] != ORC_FLUID) continue;\n        if (P->outlet_kind == ORC_OUT_CHARACTERISTIC) {',
         '        if (S->tag[i] != ORC_FLUID && S->tag[i] != ORC_OUTLET) continue;\n        if (P->outlet_kind == ORC_OUT_CHARACTERISTIC) {'),
    ],
    'no_wrap_y': [
        ('            S->y[i] = wrap(S->y0[i] + tau * S->vt[i], P->periodic_y, P->y_min, P->y_max);',
         '            S->y[i] = S->y0[i] + tau * S->vt[i];'),
    ],
    'init_advp_zero': [
        ('        S->advp[i] = S->u[i];\n        if (S->id[i] >= S->next_id)',
         '        S->advp[i] = 0.0;\n        if (S->id[i] >= S->next_id)'),
    ],
    'spawn_velocity_previous_time': [
        ('        inlet_velocity(P, ny_[k], S->t, &uin, &vin);',
         '        inlet_velocity(P, ny_[k], S->t - P->dt, &uin, &vin);'),
    ],
    'singular_threshold_loose': [
        ('    int singular = fabs(d) <= 1e-9 * fabs(M[0][0] * M[1][1] * M[2][2]);',
         '    int singular = fabs(d) <= 1e-1 * fabs(M[0][0] * M[1][1] * M[2][2]);'),
    ],
    'inlet_profile_at_current_y': [
        ('            inlet_velocity(P, S->y0[i], S->t + tau, &uin, &vin);',
         '            inlet_velocity(P, S->y0[i] + 0.5 * P->dx, S->t + tau, &uin, &vin);'),
    ],
    'pass_a_skips_walls': [
        ('    for (int i = 0; i < S->n; i++) {\n        double sw = 0.0, rho = 0.0, dx, dy;',
         '    for (int i = 0; i < S->n; i++) {\n        if (is_wall(S->tag[i])) continue;\n        double sw = 0.0, rho = 0.0, dx, dy;'),
    ],
    'probe_fluid_and_outlet': [
        ('            if (S->tag[j] != ORC_FLUID) continue;\n            double r2 = sep(P, qx[t], qy[t], S->x[j], S->y[j], &dx, &dy);',
         '            if (S->tag[j] != ORC_FLUID && S->tag[j] != ORC_OUTLET) continue;\n            double r2 = sep(P, qx[t], qy[t], S->x[j], S->y[j], &dx, &dy);'),
    ],
    'blue_adv_ignores_red_flag': [
        ('            } else if (S->tag[j] == ORC_OUTLET && S->redp[j]) {',
         '            } else if (S->tag[j] == ORC_OUTLET) {'),
    ],
    'gate_sample_p_only': [
        ('            rg[3 * k + 0] = S->u[i];\n            rg[3 * k + 1] = S->v[i];\n            rg[3 * k + 2] = S->p[i];\n            S->rpos[i] = (k + 1) % P->n_avg;',
         '            rg[3 * k + 2] = S->p[i];\n            S->rpos[i] = (k + 1) % P->n_avg;'),
    ],
    # ---- inlet signals' amplitudes and signs, records, window fill, length scales
    'pulse_amplitude_half': [
        ('*u += q[0] * cos(M_PI * (y - P->inlet_y0) / 12.0)',
         '*u += 0.5 * q[0] * cos(M_PI * (y - P->inlet_y0) / 12.0)'),
    ],
    'vortex_G_u_sign': [
        ('        *u = P->U + q[0] * yr / den;',
         '        *u = P->U - q[0] * yr / den;'),
    ],
    'ramp_half': [
        ('        *u = P->U * (t < q[0] ? t / q[0] : 1.0);',
         '        *u = P->U * (t < q[0] ? 0.5 * t / q[0] : 1.0);'),
    ],
    'I_thr_q_full': [
        ('    double q = 0.5 * P->rho0 * P->U * P->U;\n    return q * q',
         '    double q = P->rho0 * P->U * P->U;\n    return q * q'),
    ],
    'n_active_before_spawn': [
        ('    H->n_active = S->n;',
         '    H->n_active = S->n - made;'),
    ],
    'n_delete_zero': [
        ('    H->n_delete = ndel;',
         '    H->n_delete = 0;'),
    ],
    'vortex_xr_sign': [
        ('        double xr = P->U * (q[2] - t), yr = y - q[3];',
         '        double xr = P->U * (t - q[2]), yr = y - q[3];'),
    ],
    'modes_H': [
        ('sin((double)(k + 1) * M_PI * (y - P->inlet_y0) / P->inlet_h)',
         'sin((double)(k + 1) * M_PI * (y - P->inlet_y0) / (2.0 * P->inlet_h))'),
    ],
    'ring_fill_p_zero': [
        ('        rg[3 * k + 2] = S->p[i];\n    }\n    S->rpos[i] = 0;',
         '        rg[3 * k + 2] = 0.0;\n    }\n    S->rpos[i] = 0;'),
    ],
    'ubar_from_u_at_fill': [
        ('    S->pbar[i] = S->p[i];\n    S->J2[i] = 0.0;\n}',
         '    S->pbar[i] = 0.0;\n    S->J2[i] = 0.0;\n}'),
    ],
    'edac_h_in_nu': [
        ('    const double nu_edac = P->alpha * h * P->cs / 8.0;',
         '    const double nu_edac = P->alpha * P->dx * P->cs / 8.0;'),
    ],
    'eh2_uses_dx': [
        ('    const double eh2 = P->eta_reg * h * h;',
         '    const double eh2 = P->eta_reg * P->dx * P->dx;'),
    ],
    # ---- velocities each term takes, event order, stage lengths, more p~ and c_ij forms
    'A_j_uses_u_i': [
        ('            double Ajx = Aj * S->u[j], Ajy = Aj * S->v[j];',
         '            double Ajx = Aj * S->u[i], Ajy = Aj * S->v[i];'),
    ],
    'div_uses_transport_velocity': [
        ('            sp_rate += (S->m[j] * rhoi / rhoj) * c2 * (uij * gx + vij * gy)',
         '            sp_rate += (S->m[j] * rhoi / rhoj) * c2 * ((S->ut[i] - S->ut[j]) * gx + (S->vt[i] - S->vt[j]) * gy)'),
    ],
    'visc_uses_transport_velocity': [
        ('                sx += cij * (-ptil * gx + visc * uij);\n                sy += cij * (-ptil * gy + visc * vij);\n                continue;',
         '                sx += cij * (-ptil * gx + visc * (S->ut[i] - S->u[j]));\n                sy += cij * (-ptil * gy + visc * (S->vt[i] - S->v[j]));\n                continue;'),
    ],
    'events_kinds_reordered': [
        ('        if (k < nd) {\n            e[1] = 0; e[2] = del[k].id; e[3] = 0;',
         '        if (k < nd) {\n            e[1] = 0; e[2] = del[nd - 1 - k].id; e[3] = 0;'),
    ],
    'mirror_outlet_v_from_u': [
        ('        S->v[o] = fo[3 * t + 2];',
         '        S->v[o] = fo[3 * t + 1];'),
    ],
    'inlet_stage_x_dt': [
        ('            S->x[i] = S->x0[i] + tau * uin;\n',
         '            S->x[i] = S->x0[i] + P->dt * uin;\n'),
    ],
    'ptil_pavg_of_j': [
        ('double ptil = (rhoj * (S->p[i] - pavg) + rhoi * (S->p[j] - pavg)) / (rhoi + rhoj);',
         'double ptil = (rhoj * (S->p[i] - pavg) + rhoi * (S->p[j])) / (rhoi + rhoj);'),
    ],
    'cij_vi_only': [
        ('            double cij = Vi * Vi + Vj * Vj;',
         '            double cij = 2.0 * Vi * Vi;'),
    ],
    'edac_diffusion_gdotr_abs': [
        ('+ (cij / mi) * etile * (S->p[i] - S->p[j]) * gdotr / (r2 + eh2);',
         '+ (cij / mi) * etile * (S->p[i] - S->p[j]) * fabs(gdotr) / (r2 + eh2);'),
    ],
    'wall_p_gravity_term': [
        ('                pw = sp / sw;',
         '                pw = sp / sw + P->gx;'),
    ],
    'outlet_ut_zero': [
        ('        S->ut[o] = S->u[o];\n        S->vt[o] = S->v[o];\n    }\n    for (int o = 0; o < n; o++) {',
         '        S->ut[o] = 0.0;\n        S->vt[o] = S->v[o];\n    }\n    for (int o = 0; o < n; o++) {'),
    ],
    'mass_in_abg': [
        ('            S->abu[i] = -P->pb / mi * bx;\n            S->abv[i] = -P->pb / mi * by;',
         '            S->abu[i] = -P->pb * bx;\n            S->abv[i] = -P->pb * by;'),
    ],
}

# Mistakes with no observable effect: the forces of walls not counted in the drag are zero
# by construction, so summing every wall into the force record changes nothing; and a wall's
# transport velocity is its ghost velocity, so the solid force's viscous term cannot tell them
# apart.
EQUIVALENT = {"drag_all_walls", "visc_uses_transport_velocity"}
